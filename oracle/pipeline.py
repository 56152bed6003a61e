"""End-to-end oracle runs of the hot path (test infrastructure).

svd_path: Alg. 2 (TPC-SVD) fed by Alg. 7 (C-PWR) with re-orthonormalisation;
id_path:  Alg. 4 (TPC-ID) on the C-PWR output without re-orthonormalisation
          (the paper's ID experiments run C-PWR without it, Sec. 7).
"""
from __future__ import annotations

import numpy as np

from .sketch import sketch, subsample
from .cpwr import cpwr
from .rangefinder import range_find
from .svd import tpc_svd
from .interp import row_id


def svd_path(A, grid, k: int, q: int = 0, gram_grid=None, rtol: float = 1e-12,
             reorth: bool = True):
    Y = sketch(A, grid)
    if q > 0:
        W = subsample(A, gram_grid)
        G, _ = cpwr(Y, W, q, reorth, rtol)
    else:
        G = Y
    if q > 0 and reorth:
        # Alg. 7 with re-orthonormalisation ends with G_q <- QR(G_q): G_q already
        # has orthonormal columns, and the QR of an orthonormal matrix returns
        # its own range with no truncation (every |R_jj| = 1).
        Q, r = G, G.shape[1]
    else:
        Q, r = range_find(G, rtol)
    U, S, V, err, s_all, fro2 = tpc_svd(A, Q, k)
    return dict(Y=Y, G=G, Q=Q, r=r, U=U, S=S, V=V, err_est=err, sB=s_all, fro2=fro2)


def id_path(A, grid, k: int, q: int = 0, gram_grid=None, rtol: float = 1e-12):
    Y = sketch(A, grid)
    if q > 0:
        W = subsample(A, gram_grid)
        G, _ = cpwr(Y, W, q, False, rtol)
    else:
        G = Y
    J, P, err = row_id(G, k)
    return dict(Y=Y, G=G, J=J, P=P, err_est=err)
