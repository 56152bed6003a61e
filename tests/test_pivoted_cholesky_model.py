"""Host model of the Gram route of the rank-revealing QR(.) (Algs. 2, 3, 7 at
rtol >= 1e-6): a pivoted Cholesky of the FP64 Gram M^T M with the CPQR's
pivot, tie and stop rules, as the one-block and the left-looking GPU
factorisations run it (position order: the pivot moves to position j by the
transposition of positions j and piv).  Checked in numpy without a GPU
against the oracle's Householder CPQR.

What must hold (the reading that lets the Gram route stand in for
Householder CPQR): the remaining squared column norms of M after j
Householder steps are the diagonal of the Gram's Schur complement after j
Cholesky steps, so on inputs whose pivot choices have a clear margin the
two take the same pivots in the same order, stop at the same rank, and give
|R_jj| equal up to the Gram's rounding (~u cond(M)^2 relative to |R_00|).
"""
import numpy as np
import pytest

import oracle
import synth


def pivoted_cholesky(G, rtol, kmax=None):
    """Position-order pivoted Cholesky: R (r x c, pivoted columns), perm, r."""
    G = np.array(G, dtype=np.float64, copy=True)
    c = G.shape[0]
    kcap = c if kmax is None else min(kmax, c)
    perm = np.arange(c)
    R = np.zeros((c, c))
    top = None
    r = 0
    for j in range(kcap):
        d = np.diag(G)[j:]
        jj = int(np.argmax(d))                      # ties: lowest current position
        best = np.sqrt(max(d[jj], 0.0))
        if top is None:
            top = best
        if best == 0.0 or (j > 0 and best <= rtol * top):
            break
        piv = j + jj
        if piv != j:                                # symmetric transposition of positions j, piv
            G[[j, piv], :] = G[[piv, j], :]
            G[:, [j, piv]] = G[:, [piv, j]]
            R[:, [j, piv]] = R[:, [piv, j]]
            perm[[j, piv]] = perm[[piv, j]]
        R[j, j] = best
        R[j, j + 1:] = G[j, j + 1:] / best
        G[j + 1:, j + 1:] -= np.outer(R[j, j + 1:], R[j, j + 1:])
        r += 1
    return R[:r], perm, r


def _compare(M, rtol, kmax=None):
    gaps = []
    _, Ro, po, ro, _ = oracle.cpqr(M, kmax=kmax, rtol=rtol, gaps=gaps)
    Rc, pc, rc = pivoted_cholesky(M.T @ M, rtol, kmax)
    assert rc == ro
    assert np.array_equal(pc[:rc], po[:ro])
    scale = abs(Ro[0, 0])
    assert np.max(np.abs(np.abs(np.diag(Rc[:, :rc])) - np.abs(np.diag(Ro[:, :ro])))) <= 1e-8 * scale
    return gaps


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_same_pivots_on_clear_gap_inputs(seed):
    # columns of M = rows of a pivot-gap matrix: the CPQR of its transpose is the row ID's
    M = synth.pivot_gap_matrix(40, 300, seed=seed).T          # 300 x 40, tall-skinny
    gaps = _compare(M, rtol=0.0, kmax=30)
    assert min(gaps) > 1e-3


@pytest.mark.parametrize("rank", [5, 17])
def test_same_rank_stop_on_exact_rank_inputs(rank):
    rng = np.random.default_rng(rank)
    M = rng.standard_normal((500, rank)) @ rng.standard_normal((rank, 60))
    # the remaining norms after `rank` steps are rounding-level: both stop there
    gaps = _compare(M, rtol=1e-6)
    assert len(gaps) >= rank


def test_same_stop_on_graded_spectrum():
    # singular values 10^(-j/4): the cut at rtol = 1e-6 falls between two
    # well-separated values (no norm within a factor 10^(1/4) of the threshold)
    rng = np.random.default_rng(7)
    U, _ = np.linalg.qr(rng.standard_normal((800, 48)))
    V, _ = np.linalg.qr(rng.standard_normal((48, 48)))
    s = 10.0 ** (-np.arange(48) / 4.0 - 0.125)
    M = (U * s) @ V.T
    _compare(M, rtol=1e-6)
