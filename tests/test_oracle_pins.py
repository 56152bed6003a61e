"""Pins for the oracle's factorisations against facts the paper and the
mathematics fix (not against the oracle itself).

  * Omega = I (s = 1 injection): TPC-SVD is the exact truncated SVD, so the
    error equals Eckart-Young (Sec. 6) computed by LAPACK's SVD.
  * Exact rank-r inputs with rank(A_f D) = r are recovered to ~1e-13 and the
    singular values equal the prescribed ones (Thm. 3.2 with E_I = 0).
  * Heat field: with interior points x_p = p/(N+1) the sine modes are exactly
    orthogonal (DST-I), so sigma(A) = ((N+1)/2)^{d/2} sigma(T diag c) with
    T_{t,nu} = exp(-lambda_nu t).
  * Standard power iteration (Sec. 5): sigma((A A^T)^q A) = sigma^{2q+1};
    C-PWR with I = all columns and D = I is exactly that iteration.
  * CPQR pivots equal LAPACK dgeqp3's on inputs with a clear pivot gap.
  * Row ID: P(J,:) = I exactly; exact-rank inputs give a zero-error ID; the
    Cheng et al. existence bound sqrt(1 + k(m-k)) sigma_{k+1} holds.
  * Thm. 3.2 (TPC-SVD by the Remark): ||A - A_hat||_2 <= sigma_{k+1} + ||E_I||_2
    with E_I the residual of projecting A_f on range(A_c).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth
from synth import GridSpec


# ----------------------------------------------------------------------------
def test_omega_identity_gives_eckart_young():
    A = synth.blob_field(40, 16, 3, seed=5, kappa=1e-3, dtype="f64")     # 40 x 256
    g = GridSpec(N=(16, 16), s=(1, 1), kind="inject")
    s_ref = np.linalg.svd(A, compute_uv=False)
    for k in (1, 5, 12):
        o = oracle.svd_path(A, g, k, rtol=1e-15)
        err = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
        ey = np.sqrt(np.sum(s_ref[k:] ** 2) / np.sum(s_ref ** 2))
        assert abs(err - ey) <= 1e-12 + 1e-9 * ey
        np.testing.assert_allclose(o["S"], s_ref[:k], rtol=1e-12)
        # spectral-norm error = sigma_{k+1} (the Eckart-Young optimum of Sec. 1)
        Ah = (o["U"] * o["S"]) @ o["V"].T
        assert abs(np.linalg.norm(A - Ah, 2) - s_ref[k]) <= 1e-10 * s_ref[0]


@pytest.mark.parametrize("kind", ["inject", "fullweight", "blockavg"])
def test_exact_rank_recovered(kind):
    m, N, r = 30, 16, 6
    A, sig = synth.low_rank_matrix(m, N * N, r, seed=7, decay=0.6)
    g = GridSpec(N=(N, N), s=(2, 2), kind=kind)
    o = oracle.svd_path(A, g, r, rtol=1e-12)
    assert o["r"] == r
    np.testing.assert_allclose(o["S"], sig, rtol=1e-12)
    err = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    assert err < 1e-13
    d = oracle.id_path(A, g, r)
    assert oracle.id_rel_error(A, d["J"], d["P"]) < 1e-12


def test_heat_field_closed_form():
    m, N, K = 60, 24, 6
    A = synth.heat_field(m, N, 2, K, seed=11, dtype="f64")
    t, modes, c, lam = synth.fields.heat_params(m, 2, K, 11)
    T = np.exp(-np.outer(t, lam)) * c
    s_cf = np.linalg.svd(T, compute_uv=False) * ((N + 1) / 2.0)
    o = oracle.svd_path(A, GridSpec(N=(N, N), s=(1, 1), kind="inject"), 8, rtol=1e-15)
    np.testing.assert_allclose(o["S"], s_cf[:8], rtol=1e-10)


def test_heat_field_closed_form_3d():
    m, N, K = 20, 10, 3
    A = synth.heat_field(m, N, 3, K, seed=12, dtype="f64")
    t, modes, c, lam = synth.fields.heat_params(m, 3, K, 12)
    T = np.exp(-np.outer(t, lam)) * c
    s_cf = np.linalg.svd(T, compute_uv=False) * ((N + 1) / 2.0) ** 1.5
    s = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(s[:6], s_cf[:6], rtol=1e-10)


@pytest.mark.parametrize("q", [1, 2])
def test_cpwr_full_subsample_is_standard_power_iteration(q):
    m, n = 12, 16
    rng = np.random.default_rng(3)
    A = rng.standard_normal((m, n)) * (0.8 ** np.arange(m))[:, None]
    s = np.linalg.svd(A, compute_uv=False)
    G, _ = oracle.cpwr(A, A, q, reorth=False, rtol=0.0)
    sg = np.linalg.svd(G, compute_uv=False)
    p = s ** (2 * q + 1)
    np.testing.assert_allclose(sg[:m], p, rtol=1e-10, atol=1e-13 * p[0])
    # with re-orthonormalisation the range is the same (all of range(A) here)
    Gr, _ = oracle.cpwr(A, A, q, reorth=True, rtol=0.0)
    P1 = Gr @ np.linalg.pinv(Gr)
    U = np.linalg.svd(A)[0]
    np.testing.assert_allclose(P1, U @ U.T, atol=1e-10)


def test_cpwr_range_reorth_equals_plain_power():
    """Re-orthonormalisation changes the numbers, not the range (Sec. 5)."""
    rng = np.random.default_rng(8)
    m, n, l, k = 40, 120, 10, 10
    A = rng.standard_normal((m, n)) * (0.9 ** np.arange(n))[None, :]
    Y = A[:, :l]
    W = A[:, ::3]
    G0, _ = oracle.cpwr(Y, W, 1, reorth=False, rtol=0.0)
    G1, _ = oracle.cpwr(Y, W, 1, reorth=True, rtol=0.0)
    Q0 = np.linalg.qr(G0)[0]
    np.testing.assert_allclose(Q0 @ Q0.T, G1 @ G1.T, atol=1e-10)


def test_cpqr_pivots_match_dgeqp3():
    for seed in range(4):
        M = synth.pivot_gap_matrix(40, 25, seed=seed).T          # 25 x 40, column norms spread
        Q, R, perm, r, tail = oracle.cpqr(M, kmax=15)
        Qs, Rs, ps = sla.qr(M, pivoting=True, mode="economic")
        np.testing.assert_array_equal(perm[:15], ps[:15])
        np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(Rs))[:15], rtol=1e-12)
        np.testing.assert_allclose(Q.T @ Q, np.eye(15), atol=1e-13)
        # M[:, perm] = Q R + trailing part that lives in the orthogonal complement
        np.testing.assert_allclose(Q.T @ M[:, perm], R, atol=1e-12)


def test_cpqr_rank_stop():
    A, sig = synth.low_rank_matrix(30, 20, 7, seed=2, decay=0.5)
    Q, R, perm, r, tail = oracle.cpqr(A, rtol=1e-10)
    assert r == 7
    assert tail < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_row_id_structure_and_bound(seed):
    m, n, k = 50, 80, 8
    A = synth.blob_field(m, 9, 4, seed=seed, kappa=1e-3, dtype="f64")[:, :n]
    J, P, err = oracle.row_id(A, k)
    assert len(set(J.tolist())) == k
    assert np.array_equal(P[J], np.eye(k))                       # exact identity on J
    s = np.linalg.svd(A, compute_uv=False)
    e2 = np.linalg.norm(A - P @ A[J], 2)
    assert e2 <= np.sqrt(1 + k * (m - k)) * s[k] * (1 + 1e-9)
    # err_est is the relative Frobenius error of the ID
    assert abs(err - np.linalg.norm(A - P @ A[J]) / np.linalg.norm(A)) < 1e-12


def test_row_id_matches_dgeqp3_skeleton():
    A = synth.pivot_gap_matrix(30, 60, seed=9)
    J, P, err = oracle.row_id(A, 10)
    _, _, ps = sla.qr(A.T, pivoting=True, mode="economic")
    np.testing.assert_array_equal(J, ps[:10])


@pytest.mark.parametrize("kind", ["inject", "fullweight"])
def test_theorem_3_2_bound(kind):
    """||A_f - A_hat||_2 <= sigma_{f,k+1} + ||E_I||_2, E_I = (I - Q Q^T) A_f."""
    A = synth.blob_field(80, 32, 5, seed=4, kappa=2e-4, dtype="f64")
    g = GridSpec(N=(32, 32), s=(4, 4), kind=kind)
    s = np.linalg.svd(A, compute_uv=False)
    for k in (2, 5, 10):
        o = oracle.svd_path(A, g, k, rtol=1e-14)
        Q = o["Q"]
        EI = A - Q @ (Q.T @ A)
        lhs = np.linalg.norm(A - (o["U"] * o["S"]) @ o["V"].T, 2)
        assert lhs <= s[k] + np.linalg.norm(EI, 2) + 1e-12


def test_err_est_is_exact_projection_error():
    A = synth.blob_field(60, 16, 4, seed=6, kappa=1e-4, dtype="f64")
    g = GridSpec(N=(16, 16), s=(2, 2), kind="fullweight")
    o = oracle.svd_path(A, g, 7, rtol=1e-14)
    err = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    assert abs(err - o["err_est"]) < 1e-10
    np.testing.assert_allclose(o["U"].T @ o["U"], np.eye(7), atol=1e-12)
    np.testing.assert_allclose(o["V"].T @ o["V"], np.eye(7), atol=1e-12)


def test_cpwr_lowers_error_on_slow_decay():
    """Sec. 6-7 (qualitative): one C-PWR pass brings TPC-SVD close to the
    optimum when the sketch alone is poor (here: coarse injection of a
    field with fronts)."""
    A = synth.tanh_front_field(120, 32, 6, seed=1, dtype="f64")
    g = GridSpec(N=(32, 32), s=(8, 8), kind="inject")          # l = 16
    gi = GridSpec(N=(32, 32), s=(2, 2), kind="inject")         # |I| = 256
    k = 6
    s = np.linalg.svd(A, compute_uv=False)
    ey = np.sqrt(np.sum(s[k:] ** 2) / np.sum(s ** 2))
    e0 = oracle.svd_path(A, g, k, q=0, rtol=1e-14)
    e1 = oracle.svd_path(A, g, k, q=1, gram_grid=gi, rtol=1e-14)
    r0 = oracle.rel_fro_error(A, e0["U"], e0["S"], e0["V"]) / ey
    r1 = oracle.rel_fro_error(A, e1["U"], e1["S"], e1["V"]) / ey
    assert r1 <= r0 + 1e-12
    assert r1 < 1.5
