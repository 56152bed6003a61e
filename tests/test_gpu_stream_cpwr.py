"""C-PWR inside the single read of streamed snapshots (lrs_spc_stream_cpwr*,
Sec. 5, Alg. 7): the subsample rows W and Z^T = W^T A_f accumulate block by
block in the same pass as the sketch; the SVD takes B = M^T Z^T with the
C-PWR basis written as Q_b = W M, the row ID the iterate (W W^T)^q A_c.
Against the FP64 oracle (oracle.cpwr.single_read_svd, oracle.id_path).

Tolerances: the products are FP64, so B differs from the oracle's by FP64
rounding amplified by the conditioning of W T (the pinned bound of
tests/test_oracle_single_read.py), times 4 for the different summation
orders of the two sides; singular values by at most ||dB||_2 <= sqrt(r n)
max|dB| (Weyl); eps within the 1e-5 relative tolerance.  On the spiked
field (a clear pivot gap at every step) the skeleton is the oracle's, index
for index.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.cpwr import single_read_basis, single_read_svd
from synth import GridSpec

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


def _torch():
    import torch
    return torch


CASES = [
    # (name, m, N, s, sg, k, q, rtol, storage, push_rows, block_rows, on_device)
    ("blob_f32_q1_host", 300, 64, 4, 4, 12, 1, 1e-6, "f32", 64, 48, False),
    ("blob_f32_q2_device", 257, 64, 4, 8, 10, 2, 1e-6, "f32", 100, 100, True),
    ("blob_f64_q1_host", 200, 32, 4, 2, 10, 1, 1e-8, "f64", 37, 32, False),
]


def _run(lrs, case):
    torch = _torch()
    from paper_2105_01271_gb300 import binding
    _, m, N, s, sg, k, q, rtol, storage, push_rows, block_rows, on_device = case
    A = synth.blob_field(m, N, 5, 7, 1e-4, storage)
    grid = GridSpec((N, N), (s, s), "fullweight")
    gram = GridSpec((N, N), (sg, sg), "inject")
    prec = binding.LRS_PREC_FP64 if storage == "f64" else binding.LRS_PREC_SPLIT_BF16   # of the (unused) H^T
    st = binding.SpcStream(lrs, binding.DTYPE[storage], m, binding.grid_of(grid), block_rows, 0, prec)
    # the device case drops the SPC finishers' H^T from the pushes
    st.enable_cpwr(binding.grid_of(gram), spc_too=not on_device)
    src = torch.from_numpy(A).cuda() if on_device else torch.from_numpy(A).pin_memory()
    n = A.shape[1]
    for r0 in range(0, m, push_rows):
        b = min(push_rows, m - r0)
        st.push(src.data_ptr() + r0 * n * src.element_size(), b, n, on_device)
    U = torch.empty((m, k), dtype=torch.float64, device="cuda")
    S = torch.empty((k,), dtype=torch.float64, device="cuda")
    V = torch.empty((n, k), dtype=torch.float64, device="cuda")
    err, r, status = st.cpwr_svd(q, rtol, k, U, k, S, V, k)
    torch.cuda.synchronize()
    return st, A, grid, gram, (U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), err, r, status), src


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stream_cpwr_svd_against_the_oracle(lrs, case):
    _, m, N, s, sg, k, q, rtol, *_ = case
    st, A, grid, gram, (U, S, V, err, r, status), _ = _run(lrs, case)
    A64 = A.astype(np.float64)
    Y, W = oracle.sketch(A64, grid), oracle.subsample(A64, gram)
    Uo, So, Vo, erro, s_all, fro2, Qb = single_read_svd(A64, Y, W, k, q, rtol)
    assert r == len(s_all) and status == 0
    # the bound on dB from the conditioning of the last W T
    Qb_, M = single_read_basis(Y, W, q, rtol)
    B = M.T @ (W.T @ A64)
    kappa = np.linalg.norm(M, 2) * np.linalg.norm(W, 2)
    bound_b = 16.0 * np.sqrt(m * W.shape[1]) * U64 * kappa * np.max(np.abs(B))
    tol_s = np.sqrt(B.shape[0] * B.shape[1]) * bound_b + 64 * U64 * So[0]
    assert np.all(np.abs(S - So) <= tol_s), (np.max(np.abs(S - So)), tol_s)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
    eps_g = oracle.rel_fro_error(A64, U, S, V)
    eps_o = oracle.rel_fro_error(A64, Uo, So, Vo)
    assert abs(eps_g / eps_o - 1.0) <= 1e-5, (eps_g, eps_o)
    assert abs(err - erro) <= 1e-5 * erro
    if case[-1]:                              # no H^T kept: the SPC finisher refuses
        from paper_2105_01271_gb300 import binding
        with pytest.raises(binding.LrsError, match="no H"):
            st.svd(1e-12, k, k, 0, k, 0, 0, k)
    st.close()


def test_stream_cpwr_id_skeleton_on_a_gap_input(lrs):
    torch = _torch()
    from paper_2105_01271_gb300 import binding
    m, N, s, k, q = 300, 64, 4, 12, 1
    A, rows = synth.spiked_blob_field(m, N, 5, 7, nspikes=k, s=s, ratio=0.8, amp0=100.0, dtype="f32")
    grid = GridSpec((N, N), (s, s), "fullweight")
    gram = GridSpec((N, N), (s, s), "inject")
    d = oracle.id_path(A.astype(np.float64), grid, k, q=q, gram_grid=gram, rtol=1e-6)
    gaps = []
    oracle.row_id(d["G"], k, gaps)
    assert min(gaps[:k]) > 1e-2
    st = binding.SpcStream(lrs, binding.LRS_F32, m, binding.grid_of(grid), 64, 0, binding.LRS_PREC_SPLIT_BF16)
    st.enable_cpwr(binding.grid_of(gram))
    src = torch.from_numpy(A).pin_memory()
    st.push(src.data_ptr(), m, A.shape[1], False)
    J = torch.empty((k,), dtype=torch.int32, device="cuda")
    P = torch.empty((m, k), dtype=torch.float64, device="cuda")
    err = st.cpwr_id(q, 1e-6, k, J, P, k)
    torch.cuda.synchronize()
    assert np.array_equal(J.cpu().numpy(), d["J"])
    np.testing.assert_allclose(P.cpu().numpy(), d["P"], rtol=0, atol=1e-9)
    assert abs(err / d["err_est"] - 1.0) <= 1e-9
    st.close()


def test_stream_cpwr_validates(lrs):
    from paper_2105_01271_gb300 import binding
    st = binding.SpcStream(lrs, binding.LRS_F32, 64, binding.make_grid((16, 16), (4, 4), "fullweight"), 32, 0, 2)
    with pytest.raises(binding.LrsError, match="gram grid"):
        st.enable_cpwr(binding.make_grid((8, 8), (2, 2), "inject"))
    torch = _torch()
    U = torch.empty((64, 4), dtype=torch.float64, device="cuda")
    S = torch.empty((4,), dtype=torch.float64, device="cuda")
    V = torch.empty((256, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.LrsError, match="not called|rows pushed"):
        st.cpwr_svd(1, 1e-6, 4, U, 4, S, V, 4)
    st.close()
