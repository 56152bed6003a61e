"""End-to-end GPU parity of the hot path against the FP64 oracle.

Workloads (synth.WORKLOADS and reduced variants with the same recipe):
  * heat2d_m200_64x64_f64: FP64 data, 4x injection, k = 20, q = 0
  * a reduced blob field (600 x 128^2, FP32, full weighting s = 8, C-PWR on a
    2x injection subsample, q = 1, k = 30)

Tolerances (derived from the arithmetic, stated here):
  * FP64 path: |eps_gpu - eps_ora| <= 1e-12 and |s_i - s_i^ora| <= 1e-12 s_1
    (backward-stable FP64 steps, errors ~ m u64 ||A||).
  * FP32 path: |eps_gpu / eps_ora - 1| <= 1e-5 when eps_ora >= 1e-4 (the
    reconstruction tolerance).  Singular values per value (s_tol below): the
    entries of B = Q^T A_f carry independent zero-mean rounding errors of
    standard deviation at most c (|Q|^T |A_f|)_jk, c = c_p + (sqrt(m) + 1) u32
    (c_p the per-term error of the product form: u32, 2^-16, 2^-23), and a
    first-order change u_i^T E v_i of s_i has at most that deviation, so
    |ds_i| <= 6 c max(|Q|^T |A_f|) (six standard deviations); the tensor
    cores' truncated accumulation shrinks B by at most C_TRUNC relative (one
    FP32 ulp per MMA of an accumulation chunk), the double-float Gram adds
    2^-44 s_1^2 / s_i and the FP64 Cholesky and Jacobi 64 u64 s_1.
  * Skeleton J: identical to the oracle's wherever every pivot margin
    (best - runner-up)/best exceeds the perturbation the path's arithmetic can
    cause (FP64 sketch and CPQR: 1e-10; C-PWR products in FP32 or BF16 pieces:
    1e-2).  The generator synth.spiked_blob_field gives such margins at every
    step through C-PWR, and the tests assert it.  On the plain blob field the
    margins are not clear, so there the GPU's row ID must only be as accurate
    as the oracle's (relative 1e-3).
"""
import numpy as np
import pytest

import oracle
import synth
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


def _prefix(gaps, margin):
    n = 0
    for g in gaps:
        if g <= margin:
            break
        n += 1
    return n


# per-term error of a product form: FP32 FMA (Q rounded to FP32), two and
# three BF16 pieces
C_PIECE = {1: U32, 2: 2.0 ** -16, 3: 2.0 ** -23}
# systematic shrink of the tensor-core A-pass: each MMA's accumulation is
# truncated (less than one FP32 ulp of the running partial), and the A-pass
# accumulates 2 slabs of 64 snapshots per chunk before a round-to-nearest add:
# 16 MMAs per chunk with two pieces (stacked), 48 with three (unstacked)
C_TRUNC = {1: 0.0, 2: 16 * U32, 3: 48 * U32}


def s_tol(o, A, m, prec, values=None):
    """Per-value bound on |s_gpu - s_oracle| (module docstring) for the
    singular values `values` of B (default: S_k)."""
    QA = np.abs(o["Q"]).T @ np.abs(A)
    c = C_PIECE[prec] + (np.sqrt(m) + 1.0) * U32
    s1 = o["sB"][0]
    sv = o["S"] if values is None else np.asarray(values)
    return 6.0 * c * QA.max() + C_TRUNC[prec] * sv + 2.0 ** -44 * s1 ** 2 / sv + 64 * 2.0 ** -53 * s1


def err_est_bound2(o, A, m, prec, k):
    """Bound on |err_gpu^2 - err_oracle^2| for err^2 = sum_{i>k} s_i^2 / ||A||^2,
    from the per-value bound on the tail values."""
    tail = o["sB"][k:]
    t = s_tol(o, A, m, prec, tail)
    return float(np.sum(2.0 * tail * t + t * t) / o["fro2"])


HEAT = synth.WORKLOADS["heat2d_m200_64x64_f64"]
BLOB_SMALL = dict(m=600, N=128, grid=GridSpec((128, 128), (8, 8), "fullweight"),
                  gram=GridSpec((128, 128), (2, 2), "inject"), k=30, q=1, rtol=1e-6)
# the same field with 30 spiked snapshots: a clear pivot gap at every C-PWR ID step
SPIKE_SMALL = dict(nspikes=30, ratio=0.97, amp0=300.0)


@pytest.fixture(scope="module")
def heat():
    A = synth.make_workload(HEAT)
    return A, oracle.svd_path(A, HEAT.grid, HEAT.k, q=0, rtol=1e-14), oracle.id_path(A, HEAT.grid, HEAT.k)


@pytest.fixture(scope="module")
def blob():
    c = BLOB_SMALL
    A = synth.blob_field(c["m"], c["N"], 8, seed=1, kappa=1e-5, dtype="f32")
    o = oracle.svd_path(A, c["grid"], c["k"], q=c["q"], gram_grid=c["gram"], rtol=c["rtol"])
    d = oracle.id_path(A, c["grid"], c["k"], q=c["q"], gram_grid=c["gram"], rtol=c["rtol"])
    return A, o, d


@pytest.fixture(scope="module")
def blob_gap():
    c = BLOB_SMALL
    A, rows = synth.spiked_blob_field(c["m"], c["N"], 8, 1, s=8, kappa=1e-5, **SPIKE_SMALL)
    A64 = A.astype(np.float64)
    o = oracle.svd_path(A64, c["grid"], c["k"], q=c["q"], gram_grid=c["gram"], rtol=c["rtol"])
    d = oracle.id_path(A64, c["grid"], c["k"], q=c["q"], gram_grid=c["gram"], rtol=c["rtol"])
    return A, rows, o, d


# ---------------------------------------------------------------------------
def test_heat_svd_path(lrs, heat):
    from paper_2105_01271_gb300 import path
    A, o, _ = heat
    res = path.svd_path(lrs, _dev(A), "f64", HEAT.grid, HEAT.k, q=0, rtol=1e-14)
    assert res.r == o["r"]
    U, S, V = _np(res.U), _np(res.S), _np(res.V)
    eps_g = oracle.rel_fro_error(A, U, S, V)
    eps_o = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    assert abs(eps_g - eps_o) <= 1e-12
    assert np.all(np.abs(S - o["S"]) <= 1e-12 * o["S"][0])
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-12)
    # leading singular triplets: well separated, so vectors agree (signs fixed)
    np.testing.assert_allclose(U[:, :8], o["U"][:, :8], atol=1e-9)


def test_heat_id_path(lrs, heat):
    from paper_2105_01271_gb300 import path
    A, _, d = heat
    gaps = []
    oracle.row_id(d["G"], HEAT.k, gaps)
    res = path.id_path(lrs, _dev(A), "f64", HEAT.grid, HEAT.k, q=0)
    J, P = _np(res.J), _np(res.P)
    npre = _prefix(gaps, 1e-10)
    assert npre == HEAT.k                   # every pivot of this input is well separated
    assert np.array_equal(J, d["J"])
    assert np.array_equal(P[J], np.eye(HEAT.k))
    # C = R_11^{-1} R_12 amplifies FP64 rounding by cond(R_11) (~1e13 here):
    # |dP| <= 64 u64 cond(R_11) |P|, and the ID itself must be as accurate.
    _, R, _, _, _ = oracle.cpqr(d["G"].T, kmax=HEAT.k)
    kappa = np.linalg.cond(R[:, :HEAT.k])
    tol = 64 * 2.0 ** -53 * kappa
    assert np.all(np.abs(P - d["P"]) <= tol * np.maximum(1.0, np.abs(d["P"])))
    e_g = oracle.id_rel_error(A, J, P)
    e_o = oracle.id_rel_error(A, d["J"], d["P"])
    assert abs(e_g - e_o) <= 1e-3 * e_o + 1e-14
    assert abs(res.err_est - d["err_est"]) <= 1e-6 * d["err_est"] + 1e-15


def test_id_k_on_oracle_cpwr_sketch(lrs, blob):
    """lrs_id_k alone on the oracle's C-PWR output (FP64 input, FP64 CPQR)."""
    A, _, d = blob
    G = d["G"]
    m, l = G.shape
    k = BLOB_SMALL["k"]
    gaps = []
    Jo, Po, eo = oracle.row_id(G, k, gaps)
    torch = _torch()
    J = torch.empty((k,), dtype=torch.int32, device="cuda")
    P = torch.empty((m, k), dtype=torch.float64, device="cuda")
    err, st = lrs.id_k(_dev(G), m, l, l, k, J, P, k)
    npre = _prefix(gaps, 1e-10)
    assert npre == k
    assert np.array_equal(_np(J), Jo)
    np.testing.assert_allclose(_np(P), Po, rtol=1e-7, atol=1e-9)


# normwise accuracy of one product term per precision mode (see test_gpu_kernels):
# FP32 FMA 0, two BF16 pieces 3*2^-16, three pieces 6*2^-24
PIECE_ERR = {1: 0.0, 2: 3 * 2.0 ** -16, 3: 6 * 2.0 ** -24}


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_blob_svd_path(lrs, blob, prec):
    from paper_2105_01271_gb300 import path
    A, o, _ = blob
    c = BLOB_SMALL
    res = path.svd_path(lrs, _dev(A), "f32", c["grid"], c["k"], q=c["q"], gram=c["gram"], rtol=c["rtol"],
                        prec=prec)
    U, S, V = _np(res.U), _np(res.S), _np(res.V).astype(np.float64)
    eps_g = oracle.rel_fro_error(A, U, S, V)
    eps_o = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    assert eps_o >= 1e-4
    assert abs(eps_g / eps_o - 1.0) <= 1e-5, (eps_g, eps_o)
    tol = s_tol(o, A.astype(np.float64), c["m"], prec)
    assert np.all(np.abs(S - o["S"]) <= tol), np.max(np.abs(S - o["S"]) / tol)
    # U = Q U_B with U_B from the FP64 Jacobi: orthonormal to FP64 level
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-12)
    # err_est^2 = sum_{i>k} s_i^2 / ||A||^2: the per-value bound propagated
    b2 = err_est_bound2(o, A.astype(np.float64), c["m"], prec, c["k"])
    assert abs(res.err_est ** 2 - o["err_est"] ** 2) <= b2, (res.err_est, o["err_est"], b2)
    assert o["err_est"] <= eps_o * (1 + 1e-9)            # a lower bound of the true error


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_blob_id_path_accuracy(lrs, blob, prec):
    """The plain blob field has no clear pivot gap (its first margins are
    ~1e-5 and 0), so the skeleton is not unique at the path's precision: the
    GPU's row ID must be a valid one and as accurate as the oracle's."""
    from paper_2105_01271_gb300 import path
    A, _, d = blob
    c = BLOB_SMALL
    gaps = []
    oracle.row_id(d["G"], c["k"], gaps)
    assert _prefix(gaps, 1e-2) < c["k"]                  # no clear gap: J is not compared
    res = path.id_path(lrs, _dev(A), "f32", c["grid"], c["k"], q=c["q"], gram=c["gram"], rtol=c["rtol"],
                       prec=prec)
    J, P = _np(res.J), _np(res.P)
    assert len(set(J.tolist())) == c["k"]
    assert np.array_equal(P[J], np.eye(c["k"]))
    e_g = oracle.id_rel_error(A, J, P)
    e_o = oracle.id_rel_error(A, d["J"], d["P"])
    assert e_g <= e_o * (1 + 1e-3), (e_g, e_o)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_blob_gap_id_path(lrs, blob_gap, prec):
    """C-PWR (q = 1, FP32 or BF16-piece products) -> CPQR row ID on an input
    with a clear pivot gap at every one of the k steps: the skeleton must be
    the oracle's, index for index."""
    from paper_2105_01271_gb300 import path
    A, rows, _, d = blob_gap
    c = BLOB_SMALL
    k = c["k"]
    gaps = []
    oracle.row_id(d["G"], k, gaps)
    npre = _prefix(gaps, 1e-2)
    assert npre == k, (npre, min(gaps))
    res = path.id_path(lrs, _dev(A), "f32", c["grid"], k, q=c["q"], gram=c["gram"], rtol=c["rtol"], prec=prec)
    J, P = _np(res.J), _np(res.P)
    assert np.array_equal(J, d["J"])
    assert np.array_equal(P[J], np.eye(k))
    # C = R_11^{-1} R_12: the iterate's relative error c (products over m and
    # |I| terms, FP32 storage of W^T G) amplified by cond(R_11)
    _, R, _, _, _ = oracle.cpqr(d["G"].T, kmax=k)
    kappa = np.linalg.cond(R[:, :k])
    nI = c["gram"].l
    cp = C_PIECE[prec] + (c["m"] + nI + 4) * U32
    assert np.all(np.abs(P - d["P"]) <= 8 * cp * kappa * np.maximum(1.0, np.abs(d["P"])))
    # the ID's reconstruction error within the 1e-5 relative tolerance
    e_g = oracle.id_rel_error(A, J, P)
    e_o = oracle.id_rel_error(A, d["J"], d["P"])
    assert abs(e_g / e_o - 1.0) <= 1e-5, (e_g, e_o)
    assert abs(res.err_est / d["err_est"] - 1.0) <= 1e-5, (res.err_est, d["err_est"])


@pytest.mark.parametrize("prec", [2, 3])
def test_blob_gap_svd_path(lrs, blob_gap, prec):
    """The SVD path on the spiked field: per-value singular values, eps and the
    error estimate, with the FP64 small SVD of B."""
    from paper_2105_01271_gb300 import path
    A, _, o, _ = blob_gap
    c = BLOB_SMALL
    res = path.svd_path(lrs, _dev(A), "f32", c["grid"], c["k"], q=c["q"], gram=c["gram"], rtol=c["rtol"],
                        prec=prec)
    assert res.r == o["r"]
    U, S, V = _np(res.U), _np(res.S), _np(res.V).astype(np.float64)
    A64 = A.astype(np.float64)
    eps_g = oracle.rel_fro_error(A64, U, S, V)
    eps_o = oracle.rel_fro_error(A64, o["U"], o["S"], o["V"])
    assert eps_o >= 1e-4
    assert abs(eps_g / eps_o - 1.0) <= 1e-5, (eps_g, eps_o)
    tol = s_tol(o, A64, c["m"], prec)
    assert np.all(np.abs(S - o["S"]) <= tol), np.max(np.abs(S - o["S"]) / tol)
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-12)
    b2 = err_est_bound2(o, A64, c["m"], prec, c["k"])
    assert abs(res.err_est ** 2 - o["err_est"] ** 2) <= b2, (res.err_est, o["err_est"], b2)


# ---------------------------------------------------------------------------
# precision form on BF16 storage: the 3-D heat field (the 16.7M-dof workload's
# recipe at 64^3), 8x injection onto 8^3 (l = 512), k = 64, rtol = 2^-11
HEAT3 = dict(m=500, N=64, grid=GridSpec((64, 64, 64), (8, 8, 8), "inject"), k=64, rtol=2.0 ** -11)


@pytest.fixture(scope="module")
def heat3():
    c = HEAT3
    A = synth.heat_field(c["m"], c["N"], 3, 12, 2, "bf16")
    Ae = synth.fields.bf16_bits_to_f64(A)
    o = oracle.svd_path(Ae, c["grid"], c["k"], q=0, rtol=c["rtol"])
    d = oracle.id_path(Ae, c["grid"], c["k"], q=0, rtol=c["rtol"])
    return A, Ae, o, d


@pytest.mark.parametrize("prec", [2, 3])
def test_heat3d_bf16_svd_path(lrs, heat3, prec):
    """B = Q^T A with BF16 data (one exact piece) and Q in 2 or 3 pieces.  The
    BF16 rounding floor makes eps ~1e-3 here, so eps is held to the product
    error bound: E = B_gpu - B, ||E||_F <= (c_p + (m+2) u32) || |Q|^T |A| ||_F,
    |eps_g^2 - eps_o^2| <= (2 ||E|| eps_o ||A|| + ||E||^2) / ||A||^2."""
    from paper_2105_01271_gb300 import path
    A, Ae, o, _ = heat3
    c = HEAT3
    res = path.svd_path(lrs, _dev(A), "bf16", c["grid"], c["k"], q=0, rtol=c["rtol"], prec=prec)
    assert res.r == o["r"] and c["k"] <= o["r"] <= 128
    U, S, V = _np(res.U), _np(res.S), _np(res.V).astype(np.float64)
    eps_g = oracle.rel_fro_error(Ae, U, S, V)
    eps_o = oracle.rel_fro_error(Ae, o["U"], o["S"], o["V"])
    nA = np.linalg.norm(Ae)
    cp = PIECE_ERR[prec] + (c["m"] + 2) * U32
    e_bound = cp * np.linalg.norm(np.abs(o["Q"]).T @ np.abs(Ae))
    assert abs(eps_g ** 2 - eps_o ** 2) <= (2 * e_bound * eps_o * nA + e_bound ** 2) / nA ** 2
    assert np.all(np.abs(S - o["S"]) <= e_bound + 64 * U32 * o["S"][0])
    # U = Q U_B with U_B from the FP64 Jacobi: orthonormal to FP64 level
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-12)


def test_heat3d_bf16_id_path(lrs, heat3):
    """q = 0 and injection: the sketch is an exact copy, so the FP64 CPQR sees
    the oracle's input and every one of the k pivots must match."""
    from paper_2105_01271_gb300 import path
    A, Ae, _, d = heat3
    c = HEAT3
    gaps = []
    oracle.row_id(d["G"], c["k"], gaps)
    assert _prefix(gaps, 1e-10) == c["k"]
    res = path.id_path(lrs, _dev(A), "bf16", c["grid"], c["k"], q=0, rtol=c["rtol"], prec=2)
    J, P = _np(res.J), _np(res.P)
    assert np.array_equal(J, d["J"])
    assert np.array_equal(P[J], np.eye(c["k"]))
    _, R, _, _, _ = oracle.cpqr(d["G"].T, kmax=c["k"])
    kappa = np.linalg.cond(R[:, :c["k"]])
    assert np.all(np.abs(P - d["P"]) <= 64 * 2.0 ** -53 * kappa * np.maximum(1.0, np.abs(d["P"])))
    assert abs(res.err_est - d["err_est"]) <= 1e-9 * d["err_est"]


@pytest.mark.parametrize("prec,q", [(1, 1), (2, 1), (3, 1), (2, 0)])
def test_power_pass2_equals_two_passes(lrs, blob, prec, q):
    """lrs_power_pass2 (one touch of A_f, both C-PWR iterates) gives exactly
    what lrs_power_pass gives without and with re-orthonormalisation."""
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    A, _, _ = blob
    c = BLOB_SMALL
    m, n, l = A.shape[0], A.shape[1], c["grid"].l
    Ad = _dev(A)
    g = b.grid_of(c["grid"])
    gg = b.grid_of(c["gram"]) if q > 0 else None
    f64 = dict(dtype=torch.float64, device="cuda")
    Y1, G1, Y2, G2 = (torch.full((m, l), np.nan, **f64) for _ in range(4))
    Y, G0, G = (torch.full((m, l), np.nan, **f64) for _ in range(3))
    g1 = lrs.power_pass(Ad, b.LRS_F32, m, n, g, gg, q, 0, c["rtol"], prec, Y1, l, G1, l)
    gc2 = lrs.power_pass(Ad, b.LRS_F32, m, n, g, gg, q, 1, c["rtol"], prec, Y2, l, G2, l)
    g0, gc = lrs.power_pass2(Ad, b.LRS_F32, m, n, g, gg, q, c["rtol"], prec, Y, l, G0, l, G, l)
    torch.cuda.synchronize()
    assert gc == gc2 and g0 == g1
    # q > 0: the row-Gram form of the iterate, as many columns as the basis of QR(A_f D)
    assert (g0 == l) if q == 0 else (0 < g0 <= 128)
    assert torch.equal(Y, Y1) and torch.equal(Y, Y2)
    assert torch.equal(G0[:, :g0], G1[:, :g1])
    assert torch.equal(G[:, :gc], G2[:, :gc])


def test_row_gram_form_of_the_iterate(lrs, blob):
    """The m x r form H of the ID's iterate has the row inner products of the
    iterate (W W^T)^q A_f D: H H^T against the oracle's G G^T, within the
    products' accuracy (FP32-level, relative to ||G||^2)."""
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    A, _, d = blob
    c = BLOB_SMALL
    m, n, l = A.shape[0], A.shape[1], c["grid"].l
    Y, G = (torch.full((m, l), np.nan, dtype=torch.float64, device="cuda") for _ in range(2))
    g0 = lrs.power_pass(_dev(A), b.LRS_F32, m, n, b.grid_of(c["grid"]), b.grid_of(c["gram"]), 1, 0, c["rtol"],
                        b.LRS_PREC_FP32, Y, l, G, l)
    H = _np(G)[:, :g0]
    Go = d["G"]
    GG = Go @ Go.T
    # FP32 FMA products over m and |I| terms, FP32 operands: a few hundred u32 of ||G||^2
    assert np.max(np.abs(H @ H.T - GG)) <= 256 * U32 * np.max(np.abs(GG))
    assert abs(np.linalg.norm(H) / np.linalg.norm(Go) - 1.0) <= 1e-5


@pytest.mark.parametrize("prec", [1, 2])
def test_svd_k_with_a_basis_wider_than_the_tsqr_tree(lrs, prec):
    """FP32 B with r = 200 directions (beyond the Gram route's 128 and the
    TSQR tile's 2r rows): R of B^T comes from the pivoted QR of B's FP64
    copy.  Against the FP64 SVD of Q^T A: every singular value to the
    products' accuracy relative to s_1, U orthonormal to FP64 level."""
    from paper_2105_01271_gb300 import binding as b
    torch = _torch()
    m, n, r, k = 400, 4096, 200, 40
    A, sig = synth.low_rank_matrix(m, n, 260, seed=31, decay=0.985, dtype="f32")
    A64 = A.astype(np.float64)
    Q = np.linalg.svd(A64, full_matrices=False)[0][:, :r]
    s_ref = np.linalg.svd(Q.T @ A64, compute_uv=False)
    U = torch.empty((m, k), dtype=torch.float64, device="cuda")
    S = torch.empty((k,), dtype=torch.float64, device="cuda")
    V = torch.empty((n, k), dtype=torch.float32, device="cuda")
    err, st = lrs.svd_k(_dev(A), b.LRS_F32, m, n, n, _dev(Q), r, r, k, prec, U, k, S, V, k)
    assert st == b.LRS_OK
    Sg = _np(S)
    c = C_PIECE[prec] + (np.sqrt(m) + 1.0) * U32
    assert np.max(np.abs(Sg - s_ref[:k])) <= 8 * c * s_ref[0], np.max(np.abs(Sg - s_ref[:k])) / s_ref[0]
    Ug = _np(U)
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-12)
    tail = np.sqrt(np.sum(s_ref[k:] ** 2) / np.sum(A64 * A64))
    assert abs(err - tail) <= 1e-3 * tail
