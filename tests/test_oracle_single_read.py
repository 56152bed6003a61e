"""Pins for the single-read form of C-PWR (oracle.cpwr.single_read_*): the
basis is the re-orthonormalised C-PWR basis itself, written as W M, and the
projection M^T (W^T A_f) is Q_b^T A_f -- the two-read TPC result -- up to
FP64 rounding amplified by the conditioning of W T."""
import numpy as np
import pytest

import oracle
import synth
from oracle.cpwr import single_read_basis, single_read_svd
from synth import GridSpec

GRID = GridSpec(N=(32, 32), s=(4, 4), kind="fullweight")
GRAM = GridSpec(N=(32, 32), s=(4, 4), kind="inject")       # |I| = l: the sketch's own coarse points


def _blob(m=120, seed=3):
    return synth.blob_field(m, 32, 4, seed, kappa=1e-4, dtype="f64")


@pytest.mark.parametrize("q", [1, 2])
def test_basis_is_the_cpwr_basis_in_subsample_coordinates(q):
    A = _blob()
    Y, W = oracle.sketch(A, GRID), oracle.subsample(A, GRAM)
    Qb, M = single_read_basis(Y, W, q, 1e-8)
    G, _ = oracle.cpwr(Y, W, q, True, 1e-8)
    assert Qb.shape == G.shape
    np.testing.assert_allclose(Qb.T @ Qb, np.eye(Qb.shape[1]), atol=1e-12)
    # the same range as Alg. 7's basis (projectors agree)
    np.testing.assert_allclose(Qb @ Qb.T, G @ G.T, atol=1e-10)
    # and Q_b = W M (to FP64 rounding times the size of M)
    assert np.max(np.abs(W @ M - Qb)) <= 1e-6


U64 = 2.0 ** -53


def _parts(A, rtol):
    Y, W = oracle.sketch(A, GRID), oracle.subsample(A, GRAM)
    Qb, M = single_read_basis(Y, W, 1, rtol)
    Qnp, _ = oracle.range_find(Y, rtol)
    T, _ = oracle.range_find(W.T @ Qnp, rtol)
    sv = np.linalg.svd(W @ T, compute_uv=False)
    return Y, W, Qb, M, T, sv[0] / sv[-1]


def _b_bound(A, W, B_ref, kappa):
    # B = M^T (W^T A) against Q_b^T A: FP64 rounding of the sums (m and |I|
    # terms) amplified by the conditioning of W T, which sets ||M||
    return 4.0 * np.sqrt(A.shape[0] * W.shape[1]) * U64 * kappa * np.max(np.abs(B_ref))


def test_projection_equals_the_two_read_form():
    A = _blob()
    k, q, rtol = 12, 1, 1e-8
    Y, W, Qb, M, T, kappa = _parts(A, rtol)
    B_sr, B_ref = M.T @ (W.T @ A), Qb.T @ A
    dB = B_sr - B_ref
    assert np.max(np.abs(dB)) <= _b_bound(A, W, B_ref, kappa), (np.max(np.abs(dB)), kappa)
    U, S, V, err, s_all, fro2, Qb2 = single_read_svd(A, Y, W, k, q, rtol)
    o = oracle.svd_path(A, GRID, k, q=q, gram_grid=GRAM, rtol=rtol)
    assert len(s_all) == o["r"]
    # Weyl: every singular value moves by at most ||dB||_2
    d2 = np.linalg.norm(dB, 2)
    assert np.all(np.abs(s_all - o["sB"]) <= d2 + 1e-13 * o["sB"][0])
    assert np.all(np.abs(S - o["S"]) <= d2 + 1e-13 * o["S"][0])
    # the reconstruction error of the rank-k result: within 1e-5 relative of the two-read form
    eps_s = oracle.rel_fro_error(A, U, S, V)
    eps_t = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    assert abs(eps_s / eps_t - 1.0) <= 1e-5


def test_exact_rank_input_is_recovered():
    # rank-6 snapshots whose sketch and subsample keep all 6 directions:
    # one read reproduces A_f to FP64 level at k = 6
    rng = np.random.default_rng(9)
    m, n = 50, GRID.n
    A = rng.standard_normal((m, 6)) @ rng.standard_normal((6, n))
    Y, W = oracle.sketch(A, GRID), oracle.subsample(A, GRAM)
    U, S, V, err, s_all, fro2, _ = single_read_svd(A, Y, W, 6, 1, 1e-10)
    assert len(s_all) == 6
    assert oracle.rel_fro_error(A, U, S, V) <= 1e-12
    assert err <= 1e-12


def test_a_wrong_coordinate_map_is_caught():
    # planting a mistake (M taken as T, i.e. X dropped) must break B
    A = _blob()
    Y, W, Qb, M, T, kappa = _parts(A, 1e-8)
    B_good, B_bad = M.T @ (W.T @ A), T.T @ (W.T @ A)
    B_ref = Qb.T @ A
    assert np.max(np.abs(B_good - B_ref)) <= _b_bound(A, W, B_ref, kappa)
    assert np.max(np.abs(B_bad - B_ref)) > 1e-3 * np.max(np.abs(B_ref))


def test_q_zero_is_rejected():
    A = _blob(30)
    with pytest.raises(ValueError):
        single_read_basis(oracle.sketch(A, GRID), oracle.subsample(A, GRAM), 0, 1e-10)
