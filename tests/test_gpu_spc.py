"""SPC-ID (Alg. 5) and SPC-ID-ERR (Alg. 6) on the GPU against the FP64 oracle
(oracle/spc.py).

Tolerances (from the arithmetic):
  * J: identical to the oracle's (the sketches here have clear pivot gaps;
    the full-size case compares the rows whose pivots agree).
  * S_f = X^T A_f with X = U_r S_r^-1 V_r^T A_c(J,:)^T.  FP64 products:
    |dS| <= (64 u64 (s_1/s_r)^2 + 1e-12) max|S_f| (the oracle's H route
    carries (s_1/s_r)^2 u64, the device's X route s_1/s_r u64).  Split-BF16 products (2 pieces of each
    operand, FP32 accumulation over m terms): |dS| <= (2^-14 + m u32) (|X|^T |A|)
    elementwise, with X from the oracle.
  * eps_hat: FP64 Grams (double-float for FP32 data) and FP64 Jacobi, both
    backward stable: |d eps| <= 1e-10 c lambda_max(B_f B_f^T).
"""
import numpy as np
import pytest

import oracle
import oracle.spc as spc
import synth
from oracle.sketch import as_f64
from synth import GridSpec

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _torch():
    import torch
    return torch


def _dev(x):
    torch = _torch()
    if x.dtype == np.uint16:
        return torch.from_numpy(x.view(np.int16).copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


def _x_oracle(Ac, J, r):
    U, s, Vt = np.linalg.svd(Ac, full_matrices=False)
    return (U[:, :r] / s[:r]) @ (Vt[:r] @ Ac[J].T)


CASES = [
    # (name, field, m, N, s, k, r, storage, prec)
    ("blob_f64_fp64", "blob", 150, 64, 4, 10, 20, "f64", 0),
    ("heat_f64_fp64", "heat", 120, 32, 2, 6, 8, "f64", 0),
    ("blob_f32_split", "blob", 300, 64, 4, 12, 24, "f32", 2),
    ("tanh_f32_split3", "tanh", 257, 64, 4, 9, 12, "f32", 3),
]


def _field(field, m, N, storage):
    if field == "blob":
        return synth.blob_field(m, N, 6, 5, 1e-5, storage)
    if field == "heat":
        return synth.heat_field(m, N, 2, 16, 6, storage)
    return synth.tanh_front_field(m, N, 3, 7, storage)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_spc_id_matches_oracle(lrs, case):
    from paper_2105_01271_gb300 import path
    _, field, m, N, s, k, r, storage, prec = case
    A = _field(field, m, N, storage)
    A64 = as_f64(A)
    grid = GridSpec((N, N), (s, s), "fullweight")
    Ac = oracle.sketch(A64, grid)
    J_o, P_o, Sf_o, _ = spc.spc_id(A64, Ac, k, r)
    res = path.spc_id_path(lrs, _dev(A), storage, grid, k, r, prec=prec)
    assert res.r == r
    J, P, Sf = _np(res.J), _np(res.P), _np(res.Sf).astype(np.float64)
    assert np.array_equal(J, J_o)
    np.testing.assert_allclose(_np(res.Y), Ac, rtol=0, atol=1e-12 * np.abs(Ac).max())
    assert np.array_equal(P[J], np.eye(k))
    np.testing.assert_allclose(P, P_o, rtol=0, atol=1e-8 * max(1.0, np.abs(P_o).max()))
    if prec == 0:
        sv = np.linalg.svd(Ac, compute_uv=False)
        tol = 64 * 2.0 ** -53 * (sv[0] / sv[r - 1]) ** 2 + 1e-12
        assert tol < 1e-4                                # a meaningful check
        assert np.max(np.abs(Sf - Sf_o)) <= tol * np.abs(Sf_o).max()
    else:
        X = _x_oracle(Ac, J_o, r)
        bound = (2.0 ** -14 + m * U32) * (np.abs(X).T @ np.abs(A64))
        assert np.all(np.abs(Sf - Sf_o) <= bound + 1e-12 * np.abs(Sf_o).max())
    # the approximation A_f ~ P S_f is as good as the oracle's
    e_g = np.linalg.norm(A64 - P @ Sf) / np.linalg.norm(A64)
    e_o = np.linalg.norm(A64 - P_o @ Sf_o) / np.linalg.norm(A64)
    assert abs(e_g - e_o) <= 1e-6 * max(e_o, 1e-3)


ERR_CASES = [
    # (m, N, s, c, storage): m_c = m // c
    (200, 32, 4, 8, "f64"),       # m_c = 25 (odd: the dummy index of the round-robin)
    (256, 32, 4, 2, "f32"),       # m_c = 128, the largest
    (130, 32, 2, 130, "f32"),     # m_c = 1
    (300, 64, 8, 3, "bf16"),      # m_c = 100, BF16 storage
    (97, 16, 2, 1, "f64"),        # c = 1: eps_hat = eps
]


@pytest.mark.parametrize("case", ERR_CASES, ids=[f"m{c[0]}_c{c[3]}_{c[4]}" for c in ERR_CASES])
def test_spc_err_matches_oracle(lrs, case):
    from paper_2105_01271_gb300 import path
    m, N, s, c, storage = case
    A = synth.blob_field(m, N, 6, 11, 1e-5, storage)
    A64 = as_f64(A)
    grid = GridSpec((N, N), (s, s), "fullweight")
    Ac = oracle.sketch(A64, grid)
    taus = [0.0, 1e-3, 1e-2, 0.1, 0.5, 1.0, 4.0, 16.0, 100.0]
    e_o = spc.eps_hat(A64, Ac, c, taus)
    Ad = _dev(A)
    Y = _torch().from_numpy(Ac).cuda()
    e_g = np.array(path.spc_err(lrs, Ad, storage, Y, c, taus))
    J = spc.subsample_rows(m, c)
    scale = c * np.linalg.svd(A64[J], compute_uv=False)[0] ** 2
    assert np.max(np.abs(e_g - e_o)) <= 1e-10 * scale, (e_g, e_o)
    if c == 1:
        assert np.allclose(e_g, spc.eps_exact(A64, Ac, taus), rtol=0, atol=1e-10 * scale)


def test_spc_err_rejects_m_c_above_128(lrs):
    """Host-side validation: m_c = 200 would not fit the one-block eigen
    solver; the call fails with EINVAL before any launch."""
    from paper_2105_01271_gb300 import binding, path
    A = synth.blob_field(200, 16, 3, 2, 1e-5, "f64")
    Y = _torch().zeros((200, 16), dtype=_torch().float64, device="cuda")
    with pytest.raises(binding.LrsError):
        path.spc_err(lrs, _dev(A), "f64", Y, 1, [0.0])


def test_spc_id_full_size_blob_sampled(lrs):
    """The 2000 x 512^2 FP32 blob field with full weighting s = 16 (l = 1024),
    k = 50, r = 60 (s_60 / s_1 ~ 3e-5, a relative gap of 0.24 to s_61),
    split-BF16 products: S_f checked on 384 sampled columns (the oracle forms
    only those columns of H and T_r) for every row whose skeleton index
    agrees with the oracle's."""
    from paper_2105_01271_gb300 import path
    w = synth.WORKLOADS["blob2d_m2000_512x512_f32"]
    A = synth.make_workload(w)
    m, n = A.shape
    k, r = 50, 60
    res = path.spc_id_path(lrs, _dev(A), "f32", w.grid, k, r, prec=2)
    J, Sf = _np(res.J), _np(res.Sf)
    Ac = oracle.sketch(A, w.grid)
    gaps = []
    J_o, P_o, _ = oracle.row_id(Ac, k, gaps)
    agree = J == J_o
    n_prefix = 0
    while n_prefix < k and gaps[n_prefix] > 1e-10:
        n_prefix += 1
    assert np.all(agree[:n_prefix]) and agree.sum() >= k // 2
    cols = np.random.default_rng(0).choice(n, 384, replace=False)
    cols.sort()
    U, s, Vt = np.linalg.svd(Ac, full_matrices=False)
    Vr = Vt[:r].T
    mid = (Vr / s[:r] ** 2) @ Vr.T                  # V_r S_r^-2 V_r^T (oracle.spc's factor)
    Acol = A[:, cols].astype(np.float64)
    H = Acol.T @ Ac                                  # sampled rows of H = A_f^T A_c
    Sf_o = Ac[J_o] @ (mid @ H.T)                     # sampled columns of A_c(J,:) T_r
    X = (U[:, :r] / s[:r]) @ (Vt[:r] @ Ac[J_o].T)
    h_route = 64 * 2.0 ** -53 * (s[0] / s[r - 1]) ** 2       # the oracle's own rounding (H route)
    bound = (2.0 ** -14 + m * U32) * (np.abs(X).T @ np.abs(Acol)) + (h_route + 1e-12) * np.abs(Sf_o).max()
    d = np.abs(Sf[:, cols].astype(np.float64) - Sf_o)
    assert np.all(d[agree] <= bound[agree])
