"""GPU parity of each C-ABI call against the FP64 oracle, element by element.

Tolerances come from the arithmetic of each kernel (stated per test):
  * injection is a copy: bit-exact;
  * FP64 accumulation of k terms: |err| <= k u64 sum|terms| (u64 = 2^-53);
  * FP32 products with FP32 accumulation over K terms, inputs rounded to FP32:
    |err| <= (K + 2) u32 (|X|^T |A|)  (u32 = 2^-24).
"""
import numpy as np
import pytest

import oracle
import synth
from synth import GridSpec

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
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


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("N,s,kind", [
    ((64, 64), (4, 4), "inject"), ((48, 40), (3, 5), "inject"), ((16, 8, 8), (4, 2, 2), "inject"),
    ((64, 64), (4, 4), "fullweight"), ((30, 18), (2, 3), "fullweight"), ((8, 8, 12), (2, 4, 3), "fullweight"),
    ((32, 32), (4, 2), "blockavg"), ((9, 6, 4), (3, 3, 2), "blockavg"), ((1024,), (16,), "fullweight"),
])
def test_sketch_parity(lrs, dtype, N, s, kind):
    from paper_2105_01271_gb300.binding import DTYPE, make_grid
    torch = _torch()
    m = 37                                   # ragged against every tile
    n = int(np.prod(N))
    A64 = np.random.default_rng(1).standard_normal((m, n))
    A = synth.fields._store(A64, dtype)
    g = GridSpec(N=N, s=s, kind=kind)
    ref = oracle.sketch(A, g)
    Y = torch.empty((m, g.l), dtype=torch.float64, device="cuda")
    lrs.sketch(_dev(A), DTYPE[dtype], m, n, make_grid(N, s, kind), Y, g.l)
    got = _np(Y)
    if kind == "inject":
        assert np.array_equal(got, ref)
    else:
        D = oracle.sketch_operator(g)
        bound = 27 * U64 * (np.abs(oracle.sketch.__globals__["as_f64"](A)) @ abs(D)).astype(float)
        assert np.all(np.abs(got - ref) <= bound + 1e-300)


def test_sketch_rejects_bad_grid(lrs):
    from paper_2105_01271_gb300.binding import LrsError, make_grid, LRS_EINVAL
    torch = _torch()
    A = torch.zeros((4, 64), dtype=torch.float64, device="cuda")
    Y = torch.zeros((4, 64), dtype=torch.float64, device="cuda")
    for N, s, kind in [((64,), (3,), "inject"), ((64,), (1,), "fullweight"), ((8, 8), (0, 2), "inject")]:
        with pytest.raises(LrsError) as e:
            lrs.sketch(A, 0, 4, 64, make_grid(N, s, kind), Y, 64)
        assert e.value.status == LRS_EINVAL


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (37, 300, 129), (64, 128, 16), (200, 77, 513)])
@pytest.mark.parametrize("trans", [0, 1])
def test_gemm_tn_parity(lrs, prec, M, N, K, trans):
    torch = _torch()
    rng = np.random.default_rng(M * 1000 + N + K)
    X = rng.standard_normal((K, M))
    Aa = rng.standard_normal((K, N)).astype(np.float32)
    ref = X.T @ Aa.astype(np.float64)
    shape = (N, M) if trans else (M, N)
    Cd = torch.empty(shape, dtype=torch.float64, device="cuda")
    lrs.gemm_tn(M, N, K, _dev(X), 0, M, _dev(Aa), 1, N, Cd, 1, trans, shape[1], prec)
    got = _np(Cd).T if trans else _np(Cd)
    mag = np.abs(X).T @ np.abs(Aa.astype(np.float64))
    u = U64 if prec == 0 else U32
    assert np.all(np.abs(got - ref) <= (K + 2) * u * mag + 1e-300)


# ---------------------------------------------------------------------------
def test_range_find_exact_rank(lrs):
    torch = _torch()
    A, sig = synth.low_rank_matrix(300, 120, 17, seed=3, decay=0.7)
    Qo, ro = oracle.range_find(A, 1e-12)
    Q = torch.empty((300, 120), dtype=torch.float64, device="cuda")
    r = lrs.range_find(_dev(A), 300, 120, 120, 1e-12, Q, 120)
    assert r == ro == 17
    Qg = _np(Q)[:, :r]
    np.testing.assert_allclose(Qg.T @ Qg, np.eye(r), atol=1e-13)
    np.testing.assert_allclose(Qg @ Qg.T, Qo @ Qo.T, atol=1e-11)


@pytest.mark.parametrize("m,l", [(200, 256), (333, 97), (64, 64), (600, 200), (1100, 300)])
def test_range_find_full_rank_parity(lrs, m, l):
    torch = _torch()
    G = np.random.default_rng(m + l).standard_normal((m, l))
    Qo, ro = oracle.range_find(G, 1e-12)
    kq = min(m, l)
    Q = torch.empty((m, kq), dtype=torch.float64, device="cuda")
    r = lrs.range_find(_dev(G), m, l, l, 1e-12, Q, kq)
    assert r == ro == kq
    # same Householder sequence: Q itself agrees, not only its range
    np.testing.assert_allclose(_np(Q), Qo, atol=1e-11)


@pytest.mark.parametrize("p,c", [(16384, 72), (2000, 72), (400, 100), (1000, 128)])
def test_range_find_tall_skinny_gram_route(lrs, p, c):
    """Tall-skinny inputs at rtol = 1e-6 take the pivoted-Cholesky-of-the-Gram
    route: same rank as the oracle's Householder CPQR on a spectrum that
    crosses rtol, the same range (projector distance), orthonormal columns."""
    torch = _torch()
    rng = np.random.default_rng(p + c)
    U, _ = np.linalg.qr(rng.standard_normal((p, c)))
    V, _ = np.linalg.qr(rng.standard_normal((c, c)))
    M = (U * np.logspace(0, -9, c)) @ V.T
    Qo, ro = oracle.range_find(M, 1e-6)
    Q = torch.zeros((p, c), dtype=torch.float64, device="cuda")
    r = lrs.range_find(_dev(M), p, c, c, 1e-6, Q, c)
    assert r == ro
    Qg = _np(Q)[:, :r]
    np.testing.assert_allclose(Qg.T @ Qg, np.eye(r), atol=1e-13)
    # Q_g spans the oracle's range: distances ~ u kappa(M_r) with kappa <= 1/rtol
    assert np.linalg.norm(Qg @ (Qg.T @ Qo) - Qo) <= 1e-7
    assert np.all(np.isfinite(_np(Q)))


@pytest.mark.parametrize("shape", [(600, 1024), (600, 200)])
def test_range_find_blob_sketch(lrs, shape):
    """Wide / tall smooth sketches with a fast-decaying spectrum (truncated)."""
    torch = _torch()
    A = synth.blob_field(shape[0], 128, 8, seed=1, kappa=1e-5, dtype="f32")
    Y = oracle.sketch(A, GridSpec((128, 128), (4, 4), "fullweight"))[:, :shape[1]]
    m, l = Y.shape
    Qo, ro = oracle.range_find(Y, 1e-6)
    kq = min(m, l)
    for _ in range(2):                                   # deterministic across calls
        Q = torch.empty((m, kq), dtype=torch.float64, device="cuda")
        r = lrs.range_find(_dev(Y), m, l, l, 1e-6, Q, kq)
        assert r == ro
        Qg = _np(Q)[:, :r]
        np.testing.assert_allclose(Qg.T @ Qg, np.eye(r), atol=1e-13)
        # both sides are the QR of the same pivot columns, unique up to the
        # sign of each column (the wide route's R has a positive diagonal,
        # Householder's R_jj = -sign(x_0) ||x||)
        np.testing.assert_allclose(Qg * _col_signs(Qg, Qo), Qo, atol=1e-9)


def _col_signs(Qg, Qo):
    return np.where(np.sum(Qg * Qo, axis=0) < 0.0, -1.0, 1.0)


def _spectrum_matrix(p, c, n, seed):
    """p x c matrix of rank n with singular values logspace(0, -9, n)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((p, n)))
    V, _ = np.linalg.qr(rng.standard_normal((c, n)))
    return (U * np.logspace(0, -9, n)) @ V.T


@pytest.mark.parametrize("p,c,n", [(2000, 1024, 150), (600, 1024, 120), (129, 1000, 129),
                                   (256, 2400, 160), (1000, 131, 131), (300, 700, 300)])
def test_range_find_wide_gram_route(lrs, p, c, n):
    """Wide inputs (c > 128) at rtol = 1e-6 take the left-looking pivoted
    Cholesky route (ragged column ownership: c not a multiple of the columns
    per block; p < c and p > c); ranks above 128 (the last case, rank ~200)
    fall back to Householder CPQR.  Same rank as the oracle, orthonormal Q,
    the oracle's range up to u kappa(M_r) with kappa <= 1/rtol."""
    torch = _torch()
    M = _spectrum_matrix(p, c, n, seed=p + c)
    Qo, ro = oracle.range_find(M, 1e-6)
    kq = min(p, c)
    for _ in range(2):                                   # deterministic across calls
        Q = torch.zeros((p, kq), dtype=torch.float64, device="cuda")
        r = lrs.range_find(_dev(M), p, c, c, 1e-6, Q, kq)
        assert r == ro
        Qg = _np(Q)[:, :r]
        np.testing.assert_allclose(Qg.T @ Qg, np.eye(r), atol=1e-13)
        assert np.linalg.norm(Qg @ (Qg.T @ Qo) - Qo) <= 1e-7
        np.testing.assert_allclose(Qg * _col_signs(Qg, Qo), Qo, atol=1e-7)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("m,l,k", [(120, 80, 20), (45, 200, 30), (300, 64, 64), (200, 600, 60),
                                   (1000, 96, 40), (130, 1500, 50)])
def test_id_k_pivot_gap(lrs, seed, m, l, k):
    torch = _torch()
    Y = synth.pivot_gap_matrix(m, l, seed=seed)
    Jo, Po, eo = oracle.row_id(Y, k)
    J = torch.empty((k,), dtype=torch.int32, device="cuda")
    P = torch.empty((m, k), dtype=torch.float64, device="cuda")
    err, st = lrs.id_k(_dev(Y), m, l, l, k, J, P, k)
    Jg, Pg = _np(J), _np(P)
    assert np.array_equal(Jg, Jo)                     # identical skeleton
    assert np.array_equal(Pg[Jg], np.eye(k))          # exact identity on J
    np.testing.assert_allclose(Pg, Po, rtol=1e-9, atol=1e-11)
    assert abs(err - eo) <= 1e-10 * max(eo, 1e-16) + 1e-14


# ---------------------------------------------------------------------------
def test_svd_k_fp64_exact_rank(lrs):
    from paper_2105_01271_gb300.binding import LRS_PREC_FP64
    torch = _torch()
    m, n, r = 90, 700, 12
    A, sig = synth.low_rank_matrix(m, n, r, seed=4, decay=0.6)
    Q, _ = oracle.range_find(A, 1e-12)
    U = torch.empty((m, r), dtype=torch.float64, device="cuda")
    S = torch.empty((r,), dtype=torch.float64, device="cuda")
    V = torch.empty((n, r), dtype=torch.float64, device="cuda")
    err, st = lrs.svd_k(_dev(A), 0, m, n, n, _dev(Q), r, r, r, LRS_PREC_FP64, U, r, S, V, r)
    Uo, So, Vo, eo, _, _ = oracle.tpc_svd(A, Q, r)
    np.testing.assert_allclose(_np(S), sig, rtol=1e-12)
    np.testing.assert_allclose(_np(U), Uo, atol=1e-10)
    np.testing.assert_allclose(_np(V), Vo, atol=1e-10)


# ---------------------------------------------------------------------------
# tensor-core forms of X^T A.  Splitting x into BF16 pieces leaves |x - sum| <=
# 2^-8p |x| (p pieces); with the products i + j < p kept and FP32 accumulation
# over K terms:  |err| <= (c_p + (K + 2) 2^-24) (|X|^T |A|),
# c_2 = 3 * 2^-16 (two pieces), c_3 = 6 * 2^-24 (three pieces).
TC_CASES = [
    # (M, N, K, a_dtype)
    (1, 1, 1, "f32"), (72, 300, 129, "f32"), (128, 128, 64, "f32"), (200, 77, 513, "f32"),
    (72, 4099, 2000, "f32"), (300, 260, 70, "f64"), (64, 1000, 333, "bf16"),
    (700, 72, 9000, "f32"),          # few output tiles, long K: split-K with a fixed-order reduction
    # narrow X, wide 16-B-aligned A: the TMA-staged A-pass kernel (ragged dof and snapshot tails)
    (72, 4100, 2000, "f32"), (1, 256, 3, "f32"), (250, 1000, 200, "f32"), (16, 1032, 97, "bf16"),
    (256, 384, 64, "bf16"),
]


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("M,N,K,adt", TC_CASES)
@pytest.mark.parametrize("trans,c64", [(0, 0), (1, 1)])
def test_gemm_tc_parity(lrs, prec, M, N, K, adt, trans, c64):
    from paper_2105_01271_gb300.binding import DTYPE
    torch = _torch()
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    X = rng.standard_normal((K, M)) * np.exp(rng.uniform(-3, 3, (K, 1)))
    A64 = rng.standard_normal((K, N))
    A = synth.fields._store(A64, adt)
    Ae = oracle.sketch.__globals__["as_f64"](A)
    ref = X.T @ Ae
    shape = (N, M) if trans else (M, N)
    Cd = torch.full(shape, np.nan, dtype=torch.float64 if c64 else torch.float32, device="cuda")
    lrs.gemm_tn(M, N, K, _dev(X), 0, M, _dev(A), DTYPE[adt], N, Cd, c64, trans, shape[1], prec)
    got = _np(Cd).astype(np.float64)
    got = got.T if trans else got
    mag = np.abs(X).T @ np.abs(Ae)
    cp = 3 * 2.0 ** -16 if prec == 2 else 6 * 2.0 ** -24
    out_round = 0.0 if c64 else 2.0 ** -24
    bound = (cp + (K + 2) * 2.0 ** -24 + out_round) * mag
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= bound + 1e-300), np.max(np.abs(got - ref) / (bound + 1e-300))


def test_gemm_tc_deterministic(lrs):
    torch = _torch()
    rng = np.random.default_rng(5)
    X = rng.standard_normal((700, 90))
    A = rng.standard_normal((700, 3000)).astype(np.float32)
    outs = []
    for _ in range(3):
        Cd = torch.empty((90, 3000), dtype=torch.float32, device="cuda")
        lrs.gemm_tn(90, 3000, 700, _dev(X), 0, 90, _dev(A), 1, 3000, Cd, 0, 0, 3000, 2)
        outs.append(_np(Cd))
    assert all(np.array_equal(outs[0], o) for o in outs)


def test_kernel_timing(lrs):
    """lrs_set_kernel_timing / lrs_last_kernel_ms: -1 until a timed A-pass
    call, a positive duration after one, and the product is unchanged."""
    torch = _torch()
    rng = np.random.default_rng(6)
    X = rng.standard_normal((700, 90))
    A = rng.standard_normal((700, 3000)).astype(np.float32)
    ref = torch.empty((90, 3000), dtype=torch.float32, device="cuda")
    lrs.gemm_tn(90, 3000, 700, _dev(X), 0, 90, _dev(A), 1, 3000, ref, 0, 0, 3000, 2)
    lrs.set_kernel_timing(True)
    assert lrs.last_kernel_ms() == -1.0
    Cd = torch.empty((90, 3000), dtype=torch.float32, device="cuda")
    lrs.gemm_tn(90, 3000, 700, _dev(X), 0, 90, _dev(A), 1, 3000, Cd, 0, 0, 3000, 2)
    t = lrs.last_kernel_ms()
    lrs.set_kernel_timing(False)
    assert 0.0 < t < 1000.0
    assert lrs.last_kernel_ms() == -1.0
    assert np.array_equal(_np(Cd), _np(ref))


@pytest.mark.parametrize("p,c", [(40000, 100), (70000, 128)])
def test_range_find_very_tall_wide_basis(lrs, p, c):
    """Tall-skinny range finder with many rows and a basis near the Gram
    route's 128 columns: the triangular solve's teams grow until its rows
    and R fit in shared memory.  The basis spans the input's columns
    (projector against numpy's QR) and is orthonormal to FP64 level."""
    torch = _torch()
    rng = np.random.default_rng(41)
    M = rng.standard_normal((p, c)) * (0.93 ** np.arange(c))
    Qd = torch.empty((p, c), dtype=torch.float64, device="cuda")
    r = lrs.range_find(_dev(M), p, c, c, 1e-6, Qd, c)
    assert r == c
    Q = _np(Qd)
    np.testing.assert_allclose(Q.T @ Q, np.eye(c), atol=1e-12)
    Qo = np.linalg.qr(M)[0]
    # the same range: every principal cosine between the two bases is 1
    s = np.linalg.svd(Q.T @ Qo, compute_uv=False)
    assert np.min(s) >= 1.0 - 1e-9


def test_range_find_householder_long_columns(lrs):
    """Householder route (rtol below the Gram route's 1e-6) on columns longer
    than shared memory holds (p = 30000 doubles > 200 KB): Q is formed with
    each column in global scratch; orthonormal to FP64 level, same range."""
    torch = _torch()
    p, c = 30000, 150
    rng = np.random.default_rng(43)
    M = rng.standard_normal((p, c)) * (0.95 ** np.arange(c))
    Qd = torch.empty((p, c), dtype=torch.float64, device="cuda")
    r = lrs.range_find(_dev(M), p, c, c, 1e-10, Qd, c)
    assert r == c
    Q = _np(Qd)
    np.testing.assert_allclose(Q.T @ Q, np.eye(c), atol=1e-12)
    s = np.linalg.svd(Q.T @ np.linalg.qr(M)[0], compute_uv=False)
    assert np.min(s) >= 1.0 - 1e-9


def test_range_error_resolves_small_errors(lrs):
    """lrs_range_error = sqrt(1 - ||Q^T A||^2 / ||A||^2) cancels: both squared
    norms are summed with FP64 squares, so a range error near 1e-5 (far below
    sqrt(u32) ~ 3e-4, far above sqrt(u64)) comes out to a few percent of
    itself on a wide FP32 matrix."""
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    m, n, k = 300, 65536, 20
    rng = np.random.default_rng(47)
    A = (rng.standard_normal((m, k)) @ rng.standard_normal((k, n)) +
         3e-5 * rng.standard_normal((m, n))).astype(np.float32)
    A64 = A.astype(np.float64)
    Q = np.linalg.svd(A64, full_matrices=False)[0][:, :k]
    B = Q.T @ A64
    ref = np.sqrt(max(0.0, 1.0 - np.sum(B * B) / np.sum(A64 * A64)))
    assert 1e-6 < ref < 1e-4
    err = lrs.range_error(_dev(A), b.LRS_F32, m, n, n, _dev(Q), k, k)
    assert abs(err - ref) <= 0.05 * ref, (err, ref)
