"""Single-read SPC over streamed snapshots (lrs_spc_stream_*) against the FP64
oracle (oracle/spc.py): SPC-SVD (Alg. 3), SPC-ID (Alg. 5) and SPC-ID-ERR
(Alg. 6) from one pass over row blocks pushed from host or device memory.

Tolerances (from the arithmetic, normwise):
  * the sketch rows: FP64 sums of a few stencil terms, 1e-12 of max|A_c|.
  * H^T accumulates A_c^T A_f over the blocks: ||dH||_F <= u ||A_c||_F ||A_f||_F
    with u = m u64 (FP64 products), 2^-15 + m u32 (two BF16 pieces, FP32
    sums), 2^-22 + m u32 (three pieces).  B = X^T H^T with X = V_r S_r^-1 and
    S_f = W^T H^T with W = V_r S_r^-2 V_r^T A_c(J,:)^T inherit ||X||_2 ||dH||_F
    and ||W||_2 ||dH||_F, doubled for the product's own rounding; singular
    values move by at most ||dB||_2.  The single-pass form divides by s_r
    (Alg. 3's R_c^-1), so the cases keep s_r / s_1 moderate where the products
    are not FP64: the bound stays below 3e-2 of the k-th singular value.
"""
import numpy as np
import pytest

import oracle
import oracle.spc as spc
import synth
from oracle.sketch import as_f64
from synth import GridSpec

pytestmark = pytest.mark.gpu

U32, U64 = 2.0 ** -24, 2.0 ** -53


def _torch():
    import torch
    return torch


def _field(field, m, N, storage, seed=5):
    if field == "blob":
        return synth.blob_field(m, N, 6, seed, 1e-5, storage)
    if field == "heat":
        return synth.heat_field(m, N, 2, 16, seed, storage)
    return synth.tanh_front_field(m, N, 3, seed, storage)


CASES = [
    # (name, field, m, N, s, k, r, storage, prec, push_rows, block_rows, on_device)
    ("blob_f64_fp64_host", "blob", 150, 64, 4, 10, 20, "f64", 0, 37, 32, False),
    ("blob_f32_split_device", "blob", 300, 64, 4, 6, 8, "f32", 2, 64, 64, True),
    ("blob_f32_x3_host", "blob", 300, 64, 4, 8, 12, "f32", 3, 100, 48, False),
    ("tanh_f32_fp64_host", "tanh", 257, 64, 4, 4, 6, "f32", 0, 100, 48, False),
    ("heat_bf16_fp64_host", "heat", 200, 32, 2, 4, 6, "bf16", 0, 50, 50, False),
]


def _u(prec, m):
    return {0: m * U64, 2: 2.0 ** -15 + m * U32, 3: 2.0 ** -22 + m * U32}[prec]


def _push(stream, A, push_rows, on_device):
    torch = _torch()
    m, n = A.shape
    if on_device:
        src = torch.from_numpy(A.view(np.int16) if A.dtype == np.uint16 else A).cuda()
    else:
        src = torch.from_numpy(A.view(np.int16) if A.dtype == np.uint16 else A).pin_memory()
    esz = src.element_size()
    for r0 in range(0, m, push_rows):
        b = min(push_rows, m - r0)
        stream.push(src.data_ptr() + r0 * n * esz, b, n, on_device)
    return src


def _stream(lrs, case, err_c=0):
    from paper_2105_01271_gb300 import binding
    _, field, m, N, s, k, r, storage, prec, push_rows, block_rows, on_device = case
    A = _field(field, m, N, storage)
    grid = GridSpec((N, N), (s, s), "fullweight")
    st = binding.SpcStream(lrs, binding.DTYPE[storage], m, binding.make_grid((N, N), (s, s), "fullweight"),
                           block_rows, err_c, prec)
    keep = _push(st, A, push_rows, on_device)
    return st, A, grid, keep


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stream_svd_matches_oracle(lrs, case):
    torch = _torch()
    _, field, m, N, s, k, r, storage, prec, *_ = case
    st, A, grid, keep = _stream(lrs, case)
    A64 = as_f64(A)
    n = A64.shape[1]
    Ac = oracle.sketch(A64, grid)
    l = Ac.shape[1]
    U = torch.empty((m, k), dtype=torch.float64, device="cuda")
    S = torch.empty((k,), dtype=torch.float64, device="cuda")
    V = torch.empty((n, k), dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    err = st.svd(1e-12, r, k, U, k, S, V, k)
    torch.cuda.synchronize()
    Ag = _copy_sketch(st, m, l)
    np.testing.assert_allclose(Ag, Ac, rtol=0, atol=1e-12 * np.abs(Ac).max())
    Uo, So, Vo = spc.spc_svd(A64, Ac, k, r)
    # ||dB|| from the H^T and B products
    sc = np.linalg.svd(Ac, compute_uv=False)
    dB = 2 * _u(prec, m) * np.linalg.norm(Ac) * np.linalg.norm(A64) / sc[r - 1]
    if prec != 0:
        assert dB < 3e-2 * So[-1]                               # a meaningful check
    Sg = S.cpu().numpy()
    assert np.all(np.abs(Sg - So) <= dB + 64 * U64 * So[0] * sc[0] / sc[r - 1]), (Sg, So, dB)
    Ug, Vg = U.cpu().numpy(), V.cpu().numpy().astype(np.float64)
    e_g = np.linalg.norm(A64 - (Ug * Sg) @ Vg.T) / np.linalg.norm(A64)
    e_o = np.linalg.norm(A64 - (Uo * So) @ Vo.T) / np.linalg.norm(A64)
    assert abs(e_g - e_o) <= 4 * dB / np.linalg.norm(A64) + 1e-6 * e_o
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-6 if prec == 0 else 1e-4)
    assert err >= 0.0
    st.close()


class _DeviceArray:
    """A view of raw device memory for torch (the CUDA array interface)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _copy_sketch(st, m, l):
    torch = _torch()
    ptr = st.sketch_ptr()
    assert ptr != 0
    return torch.as_tensor(_DeviceArray(ptr, (m, l)), device="cuda").clone().cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stream_id_matches_oracle(lrs, case):
    torch = _torch()
    _, field, m, N, s, k, r, storage, prec, *_ = case
    st, A, grid, keep = _stream(lrs, case)
    A64 = as_f64(A)
    n = A64.shape[1]
    Ac = oracle.sketch(A64, grid)
    J = torch.empty((k,), dtype=torch.int32, device="cuda")
    P = torch.empty((m, k), dtype=torch.float64, device="cuda")
    Sf = torch.empty((k, n), dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    st.id(1e-12, r, k, J, P, k, Sf, n)
    J_o, P_o, Sf_o, _ = spc.spc_id(A64, Ac, k, r)
    Jg, Pg, Sfg = J.cpu().numpy(), P.cpu().numpy(), Sf.cpu().numpy().astype(np.float64)
    assert np.array_equal(Jg, J_o)
    np.testing.assert_allclose(Pg, P_o, rtol=0, atol=1e-8 * max(1.0, np.abs(P_o).max()))
    Uc, sc, Vct = np.linalg.svd(Ac, full_matrices=False)
    W = (Vct[:r].T / sc[:r] ** 2) @ (Vct[:r] @ Ac[J_o].T)     # l x k
    bound = (2 * _u(prec, m) * np.linalg.norm(W, 2) * np.linalg.norm(Ac) * np.linalg.norm(A64)
             + 64 * U64 * (sc[0] / sc[r - 1]) ** 2 * np.abs(Sf_o).max())
    assert bound < 0.15 * np.abs(Sf_o).max()                # a wrong term would miss by O(1)
    assert np.max(np.abs(Sfg - Sf_o)) <= bound
    st.close()


@pytest.mark.parametrize("c", [4, 7])
def test_stream_err_matches_oracle(lrs, c):
    case = ("blob_f32_split_host", "blob", 300, 64, 4, 12, 24, "f32", 2, 41, 32, False)
    st, A, grid, keep = _stream(lrs, case, err_c=c)
    A64 = as_f64(A)
    Ac = oracle.sketch(A64, grid)
    taus = [0.0, 0.5, 4.0, 16.0, 64.0, 256.0, 1024.0]
    e_g = np.array(st.err(taus))
    e_o = spc.eps_hat(A64, Ac, c, taus)
    J = spc.subsample_rows(A64.shape[0], c)
    scale = c * np.linalg.svd(A64[J], compute_uv=False)[0] ** 2
    assert np.max(np.abs(e_g - e_o)) <= 1e-10 * scale, (e_g, e_o)
    st.close()


def test_stream_host_side_errors(lrs):
    """Pushing past m, finishing early and estimating without kept rows fail
    on the host with a status, before any launch."""
    from paper_2105_01271_gb300 import binding
    torch = _torch()
    A = synth.blob_field(20, 16, 3, 1, 1e-5, "f32")
    st = binding.SpcStream(lrs, binding.LRS_F32, 20, binding.make_grid((16, 16), (2, 2), "fullweight"), 8, 0, 2)
    src = torch.from_numpy(A).pin_memory()
    st.push(src.data_ptr(), 12, 256, False)
    U = torch.empty((20, 4), dtype=torch.float64, device="cuda")
    S = torch.empty((4,), dtype=torch.float64, device="cuda")
    V = torch.empty((256, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.LrsError):
        st.svd(1e-12, 4, 4, U, 4, S, V, 4)                  # 12 of 20 rows
    with pytest.raises(binding.LrsError):
        st.push(src.data_ptr(), 12, 256, False)             # 24 > 20
    st.push(src.data_ptr() + 12 * 256 * 4, 8, 256, False)
    with pytest.raises(binding.LrsError):
        st.err([0.0])                                       # err_c = 0: no kept rows
    st.svd(1e-12, 4, 4, U, 4, S, V, 4)
    st.close()
