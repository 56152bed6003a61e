"""Pins for the oracle's error metrics (Sec. 6: relative Frobenius error, the
Eckart-Young optimum and MREO) against closed forms, not against the oracle.

  * singular_values, both routes.  Below 4M elements it is a dense SVD; above
    it the eigenvalues of the smaller Gram (A A^T when m <= n, A^T A when
    m > n).  Pinned on the heat field, whose singular values have the DST-I
    closed form ((N+1)/2)^{d/2} sigma(T diag c), on inputs just above the
    switch in both shapes, and by the trace identity sum s_i^2 = ||A||_F^2.
  * eckart_young: the relative optimum of Eq. (Eckart-Young) for matrices
    built as U diag(sigma) V^T with orthonormal U, V, where sigma is known by
    construction, and for the heat field's closed-form spectrum.
  * mreo: the definition evaluated by hand on a small table, and MREO = 1 for
    the truncated SVD itself (the "oracle solution" of Sec. 6).
"""
import numpy as np
import pytest

import oracle
import synth
from synth import GridSpec


def _heat_closed_form(m, N, d, K, seed):
    t, modes, c, lam = synth.fields.heat_params(m, d, K, seed)
    T = np.exp(-np.outer(t, lam)) * c
    return np.linalg.svd(T, compute_uv=False) * ((N + 1) / 2.0) ** (d / 2.0)


@pytest.mark.parametrize("m,N", [(70, 240), (4200, 32)])
def test_singular_values_gram_route_matches_closed_form(m, N):
    # m * N^2 is just above the 4M-element switch: (70, 240) has m < n and
    # takes A A^T; (4200, 32) has m > n and takes A^T A
    K, seed = 5, 21
    A = synth.heat_field(m, N, 2, K, seed=seed, dtype="f64")
    assert A.size > 4_000_000
    s = oracle.singular_values(A)
    assert len(s) == min(A.shape)
    assert np.all(np.diff(s) <= 0.0)                         # non-increasing
    s_cf = _heat_closed_form(m, N, 2, K, seed)
    # the Gram squares the spectrum: eigenvalue errors ~ c u64 s_1^2, so
    # s_i carries a relative error ~ c u64 (s_1 / s_i)^2; compare the values
    # above 1e-5 s_1 at 1e-5 relative (c u64 1e10 ~ 1e-5 with c ~ 1e4)
    keep = s_cf > 1e-5 * s_cf[0]
    assert keep.sum() >= 5
    np.testing.assert_allclose(s[:keep.sum()], s_cf[keep], rtol=1e-5)
    # the leading value is squared-conditioning-free: near u64
    assert abs(s[0] / s_cf[0] - 1.0) <= 1e-12
    # trace identity: the squares sum to ||A||_F^2 (no value lost or doubled)
    assert abs(np.sum(s ** 2) / np.sum(A * A) - 1.0) <= 1e-12
    # the rank is the number of modes: everything past K^2 is rounding noise
    assert s[K * K] <= 1e-6 * s[0]


def test_singular_values_dense_route_matches_closed_form():
    m, N, K, seed = 50, 20, 4, 22
    A = synth.heat_field(m, N, 2, K, seed=seed, dtype="f64")
    assert A.size <= 4_000_000
    s = oracle.singular_values(A)
    s_cf = _heat_closed_form(m, N, 2, K, seed)
    np.testing.assert_allclose(s[:K * K], s_cf[:K * K], rtol=1e-10, atol=1e-13 * s_cf[0])


@pytest.mark.parametrize("m,n", [(40, 300), (3000, 1500)])
def test_eckart_young_of_prescribed_spectrum(m, n):
    # A = U diag(sigma) V^T with sigma_i = 0.7^i: the optimum is known exactly
    r = 12
    A, sig = synth.low_rank_matrix(m, n, r, seed=23, decay=0.7)
    for k in (1, 4, 11):
        ey = oracle.eckart_young(A, k)
        ref = np.sqrt(np.sum(sig[k:] ** 2) / np.sum(sig ** 2))
        assert abs(ey - ref) <= 1e-9 * ref, (k, ey, ref)
    # k at the rank: the optimum is zero (rounding only)
    assert oracle.eckart_young(A, r) <= 1e-7


def test_eckart_young_is_the_truncated_svd_error():
    # the optimum is attained: the rank-k truncated SVD's relative error
    # (rel_fro_error) equals eckart_young for every k
    A = synth.heat_field(60, 16, 2, 6, seed=24, dtype="f64")
    Ub, s, Vt = np.linalg.svd(A, full_matrices=False)
    s_cf = _heat_closed_form(60, 16, 2, 6, 24)
    for k in (1, 3, 6):
        e = oracle.rel_fro_error(A, Ub[:, :k], s[:k], Vt[:k].T)
        assert abs(oracle.eckart_young(A, k) - e) <= 1e-10 * e + 1e-15
        # and it agrees with the closed-form spectrum's tail
        ref = np.sqrt(np.sum(s_cf[k:] ** 2) / np.sum(s_cf ** 2))
        assert abs(oracle.eckart_young(A, k, sigma=s_cf) - ref) <= 1e-15
        assert ref > 1e-8
        assert abs(e - ref) <= 1e-6 * ref


def test_mreo_by_hand():
    # trials: errors 1.2, 3.0, 2.0 against optima 1.0, 2.0, 1.0 -> ratios
    # 1.2, 1.5, 2.0; the maximum over trials is 2.0
    assert oracle.mreo([1.2, 3.0, 2.0], [1.0, 2.0, 1.0]) == 2.0
    # one trial: the ratio itself
    assert oracle.mreo([0.5], [0.25]) == 2.0


def test_mreo_of_the_oracle_solution_is_one():
    # Omega = I (s = 1 injection) makes TPC-SVD the truncated SVD: MREO = 1
    A = synth.blob_field(30, 16, 3, seed=25, kappa=1e-3, dtype="f64")
    g = GridSpec(N=(16, 16), s=(1, 1), kind="inject")
    errs, opt = [], []
    for k in (2, 5, 9):
        o = oracle.svd_path(A, g, k, rtol=1e-15)
        errs.append(oracle.rel_fro_error(A, o["U"], o["S"], o["V"]))
        opt.append(oracle.eckart_young(A, k))
    assert abs(oracle.mreo(errs, opt) - 1.0) <= 1e-9
    # a sketch that loses directions (8x injection, rank 4 basis) is worse
    g8 = GridSpec(N=(16, 16), s=(8, 8), kind="inject")
    o = oracle.svd_path(A, g8, 3, rtol=1e-15)
    e8 = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    assert oracle.mreo([e8], [oracle.eckart_young(A, 3)]) > 1.0
