"""Range finder (oracle; test infrastructure).

Paper, Alg. 2 ("Q_c <- QR(A_c)"), Alg. 3 ("Q_c, R_c <- QR(A_c)") and Alg. 7
("Q <- QR(G_q)") orthonormalise a sketch.  The paper assumes full column rank
(its Eq. for H R_c^{-1} = A_f^T Q_c); the sketches here can be rank deficient
(l >= m, or smooth fields with few modes), so the reading is the
rank-revealing form of the same QR: Householder QR with column pivoting,
stopped at the numerical rank r = number of steps before the largest remaining
column norm drops to rtol * |R_00|.  Q = first r Householder columns.
For a well-conditioned full-rank sketch (rtol below 1/cond) this spans exactly
the range of the paper's unpivoted QR.
"""
from __future__ import annotations

import numpy as np

from .cpqr import cpqr


def range_find(G: np.ndarray, rtol: float):
    """Orthonormal basis Q (m x r) of the numerical range of G (m x l)."""
    Q, R, perm, r, tail = cpqr(G, rtol=rtol)
    return Q, r
