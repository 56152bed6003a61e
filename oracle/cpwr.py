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
