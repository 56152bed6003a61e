"""Householder QR with column pivoting (oracle; test infrastructure).

Paper, Sec. 4: the row ID of a matrix comes from the rank-k column-pivoted QR
of its transpose, A^T Z ~ Q R with Z a permutation, Q orthonormal and R upper
triangular.  The same pivoted factorisation serves as the rank-revealing
"QR(.)" of Algs. 2, 3 and 7 when the sketch is rank deficient.

Readings:
  * Householder reflections (not modified Gram-Schmidt); every step recomputes
    the norms of all remaining columns from scratch (no down-dating).
  * Pivot = the remaining column of largest 2-norm; ties go to the lowest
    column index (numpy.argmax returns the first maximum).
  * Reflector convention (LAPACK dlarfg): for x = M[j:, j], R_jj = -sign(x_0)||x||
    with sign(0) = +1.
  * Stopping: after ``kmax`` steps, or before step j when the largest remaining
    column norm is <= rtol * |R_00| (the numerical rank).
"""
from __future__ import annotations

import numpy as np


def cpqr(M: np.ndarray, kmax: int | None = None, rtol: float = 0.0, gaps: list | None = None):
    """Pivoted Householder QR of M (p x c).

    Returns (Q, R, perm, r, tail) with r steps taken:
      Q    (p x r) orthonormal,
      R    (r x c) upper trapezoidal in pivoted column order,
      perm (c,)    M[:, perm] ~ Q R  (first r entries are the pivots),
      tail         Frobenius norm of the unreduced trailing block after r steps.
    If ``gaps`` is a list, the relative margin (best - runner-up) / best of the
    pivot choice at every step is appended to it.
    """
    M = np.array(M, dtype=np.float64, copy=True)
    p, c = M.shape
    kcap = min(p, c) if kmax is None else min(int(kmax), p, c)
    perm = np.arange(c)
    vs, r, top = [], 0, None
    for j in range(kcap):
        norms = np.sqrt(np.sum(M[j:, j:] ** 2, axis=0))
        jj = int(np.argmax(norms))
        if gaps is not None:
            rest = np.delete(norms, jj)
            gaps.append(float((norms[jj] - rest.max()) / norms[jj]) if len(rest) and norms[jj] > 0 else 1.0)
        if top is None:
            top = norms[jj]
        if norms[jj] == 0.0 or (j > 0 and norms[jj] <= rtol * top):
            break
        piv = j + jj
        if piv != j:
            M[:, [j, piv]] = M[:, [piv, j]]
            perm[[j, piv]] = perm[[piv, j]]
        x = M[j:, j].copy()
        alpha = np.linalg.norm(x)
        sgn = 1.0 if x[0] >= 0.0 else -1.0
        v = x
        v[0] += sgn * alpha                       # v = x + sign(x0)||x|| e1
        vn = np.linalg.norm(v)
        v /= vn
        M[j:, j:] -= 2.0 * np.outer(v, v @ M[j:, j:])
        M[j + 1:, j] = 0.0
        vs.append(v)
        r += 1
    R = np.triu(M[:r, :])
    Q = np.zeros((p, r))
    Q[:r, :r] = np.eye(r)
    for j in reversed(range(r)):
        v = vs[j]
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    tail = float(np.sqrt(np.sum(M[r:, r:] ** 2))) if r < min(p, c) else 0.0
    return Q, R, perm, r, tail
