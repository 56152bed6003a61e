"""TPC-SVD projection and small SVD (oracle; test infrastructure).

Paper, Sec. 3.1, Alg. 2 (after Halko et al.): with Q an orthonormal basis of
the (power-iterated) sketch,
    B = Q^T A_f,   B = U S V^T (SVD),   U <- Q U,
    U_k = U(:, 1:k), S_k = S(1:k, 1:k), V_k = V(:, 1:k).
The rank-k approximation is A_f ~ U_k S_k V_k^T.

Sign convention (a reading; the paper fixes none): each column of U_k has its
largest-magnitude entry positive, and V_k's column flips with it.

Error estimate (a reading; the paper defines none for the SVD): with the
orthonormal factor U_k = Q U_B,k the approximation is the orthogonal
projection U_k U_k^T A_f, and
  ||A_f - A_hat||_F^2 = ||(I - Q Q^T) A_f||_F^2 + sum_{i>k} s_i(B)^2 .
err_est keeps the second term, the energy of B beyond rank k, relative to
||A_f||_F^2:  err_est = sqrt(sum_{i>k} s_i^2 / ||A_f||_F^2).  It is computed
from the tail singular values directly (no cancellation against ||A_f||^2),
equals the relative Frobenius error when range(Q) holds A_f (E_I = 0 in
Thm. 3.2) and is a lower bound otherwise.
"""
from __future__ import annotations

import numpy as np

from .sketch import as_f64


def sign_fix(U: np.ndarray, V: np.ndarray):
    idx = np.argmax(np.abs(U), axis=0)
    sgn = np.sign(U[idx, np.arange(U.shape[1])])
    sgn[sgn == 0] = 1.0
    return U * sgn, V * sgn


def project(A: np.ndarray, Q: np.ndarray, col_block: int = 1 << 16):
    """B = Q^T A_f (r x n) and ||A_f||_F^2, streaming column slabs of A."""
    m, n = A.shape
    B = np.empty((Q.shape[1], n))
    fro2 = 0.0
    for c0 in range(0, n, col_block):
        blk = as_f64(A[:, c0:c0 + col_block])
        B[:, c0:c0 + blk.shape[1]] = Q.T @ blk
        fro2 += float(np.sum(blk * blk))
    return B, fro2


def svd_of_projection(B: np.ndarray, Q: np.ndarray, k: int, fro2: float):
    Ub, s, Vbt = np.linalg.svd(B, full_matrices=False)
    kk = min(k, len(s))
    U = Q @ Ub[:, :kk]
    V = Vbt[:kk].T
    U, V = sign_fix(U, V)
    S = s[:kk]
    err = float(np.sqrt(np.sum(s[kk:] ** 2) / fro2)) if fro2 > 0 else 0.0
    return U, S, V, err, s


def tpc_svd(A: np.ndarray, Q: np.ndarray, k: int):
    """Alg. 2 from a given basis Q.  Returns U (m x k), S (k), V (n x k),
    err_est, the full spectrum of B, and ||A_f||_F^2."""
    B, fro2 = project(A, Q)
    U, S, V, err, s_all = svd_of_projection(B, Q, k, fro2)
    return U, S, V, err, s_all, fro2
