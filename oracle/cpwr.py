"""Coarse-grid power iteration C-PWR (oracle; test infrastructure).

Paper, Sec. 5, Alg. 7: with W = A_f(:, I) a column subsample (|I| > k),
    Q_np <- QR(A_f D);  G <- A_f D
    repeat q times:  G <- W^T G; (optional) G <- QR(G);
                     G <- W G;   (optional) G <- QR(G)
so that range(G) approximates range((tau W W^T)^q A_f D); tau only rescales
G and leaves its range unchanged, so it is not applied here.

Readings:
  * "QR(.)" is the rank-revealing range finder (rangefinder.py) with the same
    rtol everywhere.
  * With re-orthonormalisation on, the loop starts from Q_np (the basis the
    algorithm computes anyway) instead of A_f D.  Both have the same range up
    to the directions that the rank truncation drops (below rtol of the
    largest), so the result differs only in those directions.
  * Without re-orthonormalisation the loop starts from A_f D, as printed.
"""
from __future__ import annotations

import numpy as np

from .rangefinder import range_find


def cpwr(Y: np.ndarray, W: np.ndarray, q: int, reorth: bool, rtol: float):
    """Return (G_q, Q_np).  Y = A_f D (m x l), W = A_f(:, I) (m x |I|)."""
    Qnp, _ = range_find(Y, rtol)
    G = Qnp if (reorth and q > 0) else Y.copy()
    for _ in range(q):
        G = W.T @ G
        if reorth:
            G, _ = range_find(G, rtol)
        G = W @ G
        if reorth:
            G, _ = range_find(G, rtol)
    return G, Qnp


def single_read_basis(Y: np.ndarray, W: np.ndarray, q: int, rtol: float):
    """Alg. 7 with re-orthonormalisation (q >= 1), the final basis written in
    the subsample's coordinates: returns (Q_b, M) with Q_b = QR(G_q) and
    Q_b = W M (m x r and |I| x r).

    The last iteration forms G_q = W T from the orthonormal T = QR(W^T G), so
    range(Q_b) lies in range(W T) and Q_b = W T X for the X that solves
    (W T) X = Q_b (least squares; exact since Q_b lies in that range);
    M = T X.  This is what lets B = Q_b^T A_f be formed as M^T (W^T A_f)
    from products accumulated in the same read of A_f as the sketch (reading
    of Sec. 5 for a single pass: W^T A_f is a sum over snapshot blocks, like
    A_c^T A_f in Alg. 3)."""
    if q < 1:
        raise ValueError("the single-read form needs q >= 1")
    Qnp, _ = range_find(Y, rtol)
    G = Qnp
    T = None
    for it in range(q):
        T, _ = range_find(W.T @ G, rtol)
        G = W @ T
        if it + 1 < q:
            G, _ = range_find(G, rtol)
    Qb, r = range_find(G, rtol)
    X = np.linalg.lstsq(G, Qb, rcond=None)[0]
    return Qb, T @ X


def single_read_svd(A: np.ndarray, Y: np.ndarray, W: np.ndarray, k: int, q: int, rtol: float):
    """TPC-SVD (Alg. 2) with C-PWR from one read of A_f: Z^T = W^T A_f
    (|I| x n), B = M^T Z^T = Q_b^T A_f, then SVD(B) as svd.tpc_svd.  Returns
    (U, S, V, err_est, spectrum of B, ||A_f||_F^2, Q_b)."""
    from .svd import svd_of_projection
    from .sketch import as_f64
    Af = as_f64(A)
    Qb, M = single_read_basis(Y, W, q, rtol)
    Zt = W.T @ Af
    B = M.T @ Zt
    fro2 = float(np.sum(Af * Af))
    U, S, V, err, s_all = svd_of_projection(B, Qb, k, fro2)
    return U, S, V, err, s_all, fro2, Qb
