"""Deterministic sketch operators, formed explicitly (oracle; test infrastructure).

Paper, Sec. 2 ("Deterministic sketches for low-rank approximations", Table 1):
A_c = A_f D with D (n x n_c) one of
  * direct injection       -- D_ij = 1 at the one fine point sampled for coarse j,
  * nearest neighbour      -- weights 1/4, 1/2, 1/4 on the centre and its two
                              neighbours (d = 1; the "full weighting" stencil),
  * global sketch          -- the unweighted mean 1/s over s consecutive dofs.

Readings (the paper writes D in 1-D on the vectorised index only):
  * Tensor product over grid axes, x fastest: D = D_z (x) D_y (x) D_x, so that
    A_c[:, (zc*Ncy + yc)*Ncx + xc] = sum D_z[z,zc] D_y[y,yc] D_x[x,xc] A_f[:, (z*Ny+y)*Nx+x].
  * Per axis the coarse point j (0-based) sits at fine index c_j = s*j + s//2.
    The paper's "i = js + 1" overruns n at j = n_c; the cell centre does not,
    and s = 1 gives D = I.
  * Nearest neighbour at c_j reads c_j - 1, c_j, c_j + 1.  A neighbour outside
    the grid (only possible for s = 2 at the last cell) counts as zero, with no
    renormalisation.  The stencil needs s >= 2.
  * Global sketch averages the s fine points of cell j: s*j .. s*j + s - 1
    (Table 1's stencil size "s - 1" is read as s, as the definition says).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def restriction_1d(N: int, s: int, kind: str) -> sp.csr_matrix:
    """D for one axis: N fine points -> N // s coarse points (N % s == 0)."""
    if N % s != 0:
        raise ValueError("N must be a multiple of s")
    nc = N // s
    rows, cols, vals = [], [], []
    for j in range(nc):
        c = s * j + s // 2
        if kind == "inject":
            rows.append(c); cols.append(j); vals.append(1.0)
        elif kind == "fullweight":
            if s < 2:
                raise ValueError("nearest-neighbour stencil needs s >= 2")
            for off, w in ((-1, 0.25), (0, 0.5), (1, 0.25)):
                i = c + off
                if 0 <= i < N:
                    rows.append(i); cols.append(j); vals.append(w)
        elif kind == "blockavg":
            for t in range(s):
                rows.append(s * j + t); cols.append(j); vals.append(1.0 / s)
        else:
            raise ValueError(kind)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, nc))


def sketch_operator(grid) -> sp.csr_matrix:
    """Full D (n x l) as the Kronecker product of the per-axis operators.

    ``grid`` has N (x first), s and kind (see synth.GridSpec)."""
    D = None
    for Nd, sd in zip(grid.N, grid.s):       # x, y, z
        Dd = restriction_1d(Nd, sd, grid.kind)
        D = Dd if D is None else sp.kron(Dd, D, format="csr")   # slower axis on the left
    return D.tocsr()


def as_f64(A: np.ndarray, dtype: str | None = None) -> np.ndarray:
    """Exact float64 view of stored values (bf16 given as uint16 bit patterns)."""
    if A.dtype == np.uint16:
        u = A.astype(np.uint32) << 16
        return u.view(np.float32).astype(np.float64)
    return np.asarray(A, dtype=np.float64)


def sketch(A: np.ndarray, grid, row_block: int = 256) -> np.ndarray:
    """A_c = A_f D in float64 (rows streamed in blocks, as in Alg. 3's loop)."""
    D = sketch_operator(grid)
    m = A.shape[0]
    out = np.empty((m, D.shape[1]))
    for r0 in range(0, m, row_block):
        blk = as_f64(A[r0:r0 + row_block])
        out[r0:r0 + len(blk)] = (D.T @ blk.T).T
    return out


def subsample_index(grid) -> np.ndarray:
    """Column index set I of A_f(:, I) for C-PWR (Alg. 7): the fine points that
    direct injection with the grid's factors samples, in coarse-index order."""
    S = sketch_operator(type(grid)(N=grid.N, s=grid.s, kind="inject"))
    S = S.tocsc()
    idx = np.empty(S.shape[1], dtype=np.int64)
    for j in range(S.shape[1]):
        col = S.indices[S.indptr[j]:S.indptr[j + 1]]
        assert len(col) == 1
        idx[j] = col[0]
    return idx


def subsample(A: np.ndarray, grid) -> np.ndarray:
    """A_c = A_f(:, I) (Alg. 7), float64, through the explicit selection matrix."""
    I = subsample_index(grid)
    n = A.shape[1]
    Sel = sp.csr_matrix((np.ones(len(I)), (I, np.arange(len(I)))), shape=(n, len(I)))
    return (Sel.T @ as_f64(A).T).T
