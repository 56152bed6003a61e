"""Row interpolative decomposition on the sketch (oracle; test infrastructure).

Paper, Sec. 4 and Alg. 4 (TPC-ID): the row ID  A ~ P A(I, :)  with P(I,:) = I_k
comes from the rank-k column-pivoted QR of A^T:
    A^T Z ~ Q [R_1 | R_2],   R_2 ~ R_1 C,   P = ([I | C] Z^T)^T.
TPC-ID computes (I_c, P_c) on the sketch A_c = A_f D (or on the C-PWR output
G_q) and lifts with the fine rows:  A_f ~ P_c A_f(I_c, :).

Readings:
  * The paper says "solving R_2 ~ R_1 C via least squares"; R_1 is square and
    upper triangular, so the solve is the triangular solve C = R_1^{-1} R_2.
  * I_c are snapshot (row) indices: the first k pivots of the CPQR of A_c^T.
  * err_est = ||R_22||_F / ||A_c||_F, the relative Frobenius error of the
    coarse row ID P_c A_c(I_c, :) (the unreduced trailing block of the CPQR).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .cpqr import cpqr


def row_id(Ac: np.ndarray, k: int, gaps: list | None = None):
    """Rank-k row ID of Ac (m x l).  Returns (J, P, err_est); ``gaps`` as in cpqr."""
    m = Ac.shape[0]
    _, R, perm, r, tail = cpqr(Ac.T, kmax=k, gaps=gaps)
    if r < k:
        raise ValueError(f"numerical rank {r} < k = {k}")
    R1, R2 = R[:, :k], R[:, k:]
    C = solve_triangular(R1, R2, lower=False)          # k x (m - k)
    P = np.zeros((m, k))
    P[perm[:k], :] = np.eye(k)
    P[perm[k:], :] = C.T
    nrm = np.linalg.norm(Ac)
    err = tail / nrm if nrm > 0 else 0.0
    return perm[:k].copy(), P, err


def tpc_id(Af: np.ndarray, Ac: np.ndarray, k: int):
    """Alg. 4: ID on the sketch, lifted with the fine skeleton rows."""
    J, P, err = row_id(Ac, k)
    return J, P, err, Af[J]
