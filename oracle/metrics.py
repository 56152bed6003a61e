"""Error metrics (oracle; test infrastructure).

Paper, Sec. 6: relative Frobenius error ||A_f - A_hat||_F / ||A_f||_F; the
Eckart-Young optimum ||A_f - A_{f,k}||_F = (sum_{i>k} sigma_i^2)^{1/2}; and
MREO = max over trials of ||A_f - A_hat||_F / ||A_f - A_{f,k}||_F.
"""
from __future__ import annotations

import numpy as np

from .sketch import as_f64


def rel_fro_error(A: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray,
                  col_block: int = 1 << 15) -> float:
    """||A - U diag(S) V^T||_F / ||A||_F, streaming column slabs."""
    num = den = 0.0
    US = U * S
    for c0 in range(0, A.shape[1], col_block):
        blk = as_f64(A[:, c0:c0 + col_block])
        R = blk - US @ V[c0:c0 + blk.shape[1]].T
        num += float(np.sum(R * R))
        den += float(np.sum(blk * blk))
    return float(np.sqrt(num / den))


def id_rel_error(A: np.ndarray, J: np.ndarray, P: np.ndarray, col_block: int = 1 << 15) -> float:
    """||A - P A(J,:)||_F / ||A||_F."""
    num = den = 0.0
    for c0 in range(0, A.shape[1], col_block):
        blk = as_f64(A[:, c0:c0 + col_block])
        R = blk - P @ blk[J]
        num += float(np.sum(R * R))
        den += float(np.sum(blk * blk))
    return float(np.sqrt(num / den))


def singular_values(A: np.ndarray) -> np.ndarray:
    """All singular values of A via the eigenvalues of the smaller Gram matrix
    accumulated in float64 (dense SVD for small inputs)."""
    A64 = as_f64(A)
    m, n = A64.shape
    if m * n <= 4_000_000:
        return np.linalg.svd(A64, compute_uv=False)
    G = A64 @ A64.T if m <= n else A64.T @ A64
    ev = np.linalg.eigvalsh(G)[::-1]
    return np.sqrt(np.clip(ev, 0.0, None))


def eckart_young(A: np.ndarray, k: int, sigma: np.ndarray | None = None) -> float:
    """Relative optimal rank-k Frobenius error (sum_{i>k} s_i^2 / sum s_i^2)^{1/2}."""
    s = singular_values(A) if sigma is None else np.asarray(sigma)
    s2 = s ** 2
    return float(np.sqrt(np.sum(s2[k:]) / np.sum(s2)))


def mreo(errors, optimal) -> float:
    """Max ratio of error to the Eckart-Young optimum over trials."""
    e = np.asarray(errors, dtype=np.float64)
    o = np.asarray(optimal, dtype=np.float64)
    return float(np.max(e / o))
