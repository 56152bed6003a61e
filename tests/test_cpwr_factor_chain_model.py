"""Host model of the row ID's C-PWR iterate formed from the factors of the
re-orthonormalised loop (Alg. 7 run once with QR(.) after every product;
the ID wants the iterate without re-orthonormalisation, (W W^T)^q Y), checked
in numpy FP64 without a GPU.

Every QR(.) returns its factor in original column order, input = Q Rt, so
    Y = Q_np Rt_np,  W^T Q = Q_t Rt_t,  W Q_t = Q_g Rt_g,  ...
and (W W^T)^q Y = Q_q M Rt_np with M = Rt_g,q Rt_t,q ... Rt_g,1 Rt_t,1.
With Ra^T Ra = Rt_np Rt_np^T (a Cholesky factor), H = Q_q M Ra^T (m x r_np)
has H H^T equal to the iterate's row Gram, so the CPQR of H^T (r_np rows
instead of l) picks the iterate's rows.  What must hold, on full-rank
bases (no truncation): H H^T equals D D^T for the directly formed
D = (W W^T)^q Y to FP64 rounding, and on a clear-gap input the row IDs of
H and of D pick the same k rows.
"""
import numpy as np
import pytest

import oracle


def qr_orig(M):
    """M = Q Rt with Rt in M's own column order (unpivoted QR, full rank)."""
    Q, R = np.linalg.qr(M)
    return Q, R


def chain(Y, W, q):
    Qnp, Rt_np = qr_orig(Y)
    M = None
    G = Qnp
    for _ in range(q):
        Qt, Rt_t = qr_orig(W.T @ G)
        Qg, Rt_g = qr_orig(W @ Qt)
        step = Rt_g @ Rt_t
        M = step if M is None else step @ M
        G = Qg
    Ra = np.linalg.cholesky(Rt_np @ Rt_np.T).T          # Ra^T Ra = Rt_np Rt_np^T
    return G @ M @ Ra.T


def gap_inputs(seed, m=120, l=40, nI=300, ratio=0.85):
    """A_f-like data: rows scaled geometrically so the row ID has clear
    margins; Y and W two different column samplings of it."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 2000)) * (ratio ** rng.permutation(m))[:, None]
    cols = rng.permutation(2000)
    return A[:, cols[:l]], A[:, cols[l:l + nI]]


@pytest.mark.parametrize("q", [1, 2])
def test_row_gram_identity(q):
    Y, W = gap_inputs(q)
    D = Y.copy()
    for _ in range(q):
        D = W @ (W.T @ D)
    H = chain(Y, W, q)
    assert H.shape == (Y.shape[0], Y.shape[1])
    G1, G2 = H @ H.T, D @ D.T
    assert np.max(np.abs(G1 - G2)) <= 1e-12 * np.max(np.abs(G2))


@pytest.mark.parametrize("q", [1, 2])
def test_row_id_of_the_factor_chain(q):
    Y, W = gap_inputs(10 + q)
    D = Y.copy()
    for _ in range(q):
        D = W @ (W.T @ D)
    H = chain(Y, W, q)
    k = 25
    gaps = []
    Jd, _, _ = oracle.row_id(D, k, gaps)
    assert min(gaps) > 1e-3
    Jh, _, _ = oracle.row_id(H, k)
    assert np.array_equal(Jd, Jh)
