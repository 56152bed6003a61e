"""The hot path as a sequence of C-ABI calls (orchestration only).

``svd_path`` = lrs_power_pass (sketch + C-PWR with re-orthonormalisation) ->
lrs_range_find -> lrs_svd_k  (paper Algs. 7 and 2);
``id_path``  = lrs_power_pass (C-PWR without re-orthonormalisation, as in the
paper's ID experiments) -> lrs_id_k  (Alg. 4);
``power_pass2`` + ``svd_from_pass`` / ``id_from_pass`` = both paths of one
matrix from one touch of A_f (lrs_power_pass2: the sketch and the subsample
read once, both C-PWR iterates);
``spc_id_path`` = lrs_sketch -> lrs_sketch_svd -> lrs_id_k -> lrs_spc_lift
(SPC-ID, Alg. 5); ``spc_err`` = lrs_spc_err (Alg. 6).
Device buffers come from torch; every arithmetic step runs in liblrs.so.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from .binding import (DTYPE, LRS_PREC_FP32, LRS_PREC_FP64, Context, grid_of)


@dataclass
class SvdResult:
    U: torch.Tensor
    S: torch.Tensor
    V: torch.Tensor
    err_est: float
    r: int
    g_cols: int
    status: int


@dataclass
class IdResult:
    J: torch.Tensor
    P: torch.Tensor
    err_est: float
    status: int


def default_prec(dtype: str) -> int:
    return LRS_PREC_FP64 if dtype == "f64" else LRS_PREC_FP32


class Buffers:
    """Device buffers of one decomposition, allocated once and reused."""

    def __init__(self, m, n, l, k, dev, v_f64):
        f64 = torch.float64
        self.Y = torch.empty((m, l), dtype=f64, device=dev)
        self.G = torch.empty((m, l), dtype=f64, device=dev)
        self.Q = torch.empty((m, min(m, l)), dtype=f64, device=dev)
        self.U = torch.empty((m, k), dtype=f64, device=dev)
        self.S = torch.empty((k,), dtype=f64, device=dev)
        self.V = torch.empty((n, k), dtype=f64 if v_f64 else torch.float32, device=dev)
        self.Yid = torch.empty((m, l), dtype=f64, device=dev)
        self.Gid = torch.empty((m, l), dtype=f64, device=dev)
        self.J = torch.empty((k,), dtype=torch.int32, device=dev)
        self.P = torch.empty((m, k), dtype=f64, device=dev)


def svd_path(ctx: Context, A: torch.Tensor, dtype: str, grid, k: int, q: int = 0, gram=None,
             rtol: float = 1e-12, prec: int | None = None, bufs: Buffers | None = None) -> SvdResult:
    m = A.shape[0]
    n = A.shape[1]
    dt = DTYPE[dtype]
    prec = default_prec(dtype) if prec is None else prec
    g = grid_of(grid)
    l = int(grid.l)
    gg = grid_of(gram) if (gram is not None and q > 0) else None
    b = bufs or Buffers(m, n, l, k, A.device, prec == LRS_PREC_FP64)
    gc = ctx.power_pass(A, dt, m, n, g, gg, q, 1, rtol, prec, b.Y, l, b.G, l)
    if q > 0:
        # a re-orthonormalised C-PWR pass ends with QR(G_q): G_q is the basis
        Qb, ldq, r = b.G, l, gc
    else:
        ldq = b.Q.shape[1]
        r = ctx.range_find(b.G, m, gc, l, rtol, b.Q, ldq)
        Qb = b.Q
    err, st = ctx.svd_k(A, dt, m, n, n, Qb, ldq, r, k, prec, b.U, k, b.S, b.V, k)
    kk = min(k, r)
    return SvdResult(b.U[:, :kk], b.S[:kk], b.V[:, :kk], err, r, gc, st)


def id_path(ctx: Context, A: torch.Tensor, dtype: str, grid, k: int, q: int = 0, gram=None,
            rtol: float = 1e-12, prec: int | None = None, bufs: Buffers | None = None) -> IdResult:
    m = A.shape[0]
    n = A.shape[1]
    dt = DTYPE[dtype]
    prec = default_prec(dtype) if prec is None else prec
    g = grid_of(grid)
    l = int(grid.l)
    gg = grid_of(gram) if (gram is not None and q > 0) else None
    b = bufs or Buffers(m, n, l, k, A.device, prec == LRS_PREC_FP64)
    g0 = ctx.power_pass(A, dt, m, n, g, gg, q, 0, rtol, prec, b.Yid, l, b.Gid, l)
    err, st = ctx.id_k(b.Gid, m, g0, l, k, b.J, b.P, k)
    return IdResult(b.J, b.P, err, st)


def power_pass2(ctx: Context, A: torch.Tensor, dtype: str, grid, q: int = 0, gram=None, rtol: float = 1e-12,
                prec: int | None = None, bufs: Buffers | None = None):
    """One touch of A_f for both paths: the sketch into bufs.Y, the ID's C-PWR
    iterate into bufs.Gid, the SVD's orthonormal one into bufs.G; returns
    (columns of the ID's iterate, SVD basis width)."""
    m, n = A.shape
    prec = default_prec(dtype) if prec is None else prec
    l = int(grid.l)
    gg = grid_of(gram) if (gram is not None and q > 0) else None
    return ctx.power_pass2(A, DTYPE[dtype], m, n, grid_of(grid), gg, q, rtol, prec, bufs.Y, l, bufs.Gid, l,
                           bufs.G, l)


def svd_from_pass(ctx: Context, A: torch.Tensor, dtype: str, grid, k: int, q: int, gc: int, rtol: float,
                  prec: int, bufs: Buffers) -> SvdResult:
    """The SVD path after power_pass2 (the basis of bufs.G, gc columns: the
    second value power_pass2 returns)."""
    m, n = A.shape
    l = int(grid.l)
    if q > 0:
        Qb, ldq, r = bufs.G, l, gc
    else:
        ldq = bufs.Q.shape[1]
        r = ctx.range_find(bufs.G, m, gc, l, rtol, bufs.Q, ldq)
        Qb = bufs.Q
    err, st = ctx.svd_k(A, DTYPE[dtype], m, n, n, Qb, ldq, r, k, prec, bufs.U, k, bufs.S, bufs.V, k)
    kk = min(k, r)
    return SvdResult(bufs.U[:, :kk], bufs.S[:kk], bufs.V[:, :kk], err, r, gc, st)


def id_from_pass(ctx: Context, m: int, grid, k: int, g0: int, bufs: Buffers) -> IdResult:
    """The row ID after power_pass2 (the iterate in bufs.Gid, g0 columns: the
    first value power_pass2 returns)."""
    l = int(grid.l)
    err, st = ctx.id_k(bufs.Gid, m, g0, l, k, bufs.J, bufs.P, k)
    return IdResult(bufs.J, bufs.P, err, st)


@dataclass
class SpcResult:
    J: torch.Tensor
    P: torch.Tensor
    Sf: torch.Tensor       # lifted skeleton A_c(J,:) T_r (k x n): A_f ~ P Sf
    Y: torch.Tensor        # the sketch A_c
    U: torch.Tensor        # leading r singular triplets of A_c
    S: torch.Tensor
    V: torch.Tensor
    r: int                 # lifting rank used
    rank_c: int            # numerical rank of the sketch
    err_est: float         # coarse ID error (lrs_id_k)
    status: int


def spc_id_path(ctx: Context, A: torch.Tensor, dtype: str, grid, k: int, r_lift: int, rtol: float = 1e-12,
                prec: int | None = None) -> SpcResult:
    """SPC-ID (Alg. 5): the sketch, its leading r triplets (r = r_lift, at
    most the sketch's numerical rank at rtol), the row ID of the sketch, and
    the lifted skeleton from one read of A_f."""
    m, n = A.shape
    dt = DTYPE[dtype]
    prec = default_prec(dtype) if prec is None else prec
    l = int(grid.l)
    dev = A.device
    f64 = torch.float64
    Y = torch.empty((m, l), dtype=f64, device=dev)
    ctx.sketch(A, dt, m, n, grid_of(grid), Y, l)
    ldq = min(m, l)
    Q = torch.empty((m, ldq), dtype=f64, device=dev)
    r = int(r_lift)
    U = torch.empty((m, r), dtype=f64, device=dev)
    S = torch.empty((r,), dtype=f64, device=dev)
    V = torch.empty((l, r), dtype=f64, device=dev)
    rank_c = ctx.sketch_svd(Y, m, l, l, rtol, Q, ldq, r, U, r, S, V, r)
    J = torch.empty((k,), dtype=torch.int32, device=dev)
    P = torch.empty((m, k), dtype=f64, device=dev)
    err, st = ctx.id_k(Y, m, l, l, k, J, P, k)
    Sf = torch.empty((k, n), dtype=f64 if prec == LRS_PREC_FP64 else torch.float32, device=dev)
    ctx.spc_lift(A, dt, m, n, n, Y, l, l, U, r, S, V, r, r, J, k, prec, Sf, n)
    return SpcResult(J, P, Sf, Y, U, S, V, r, rank_c, err, st)


def spc_err(ctx: Context, A: torch.Tensor, dtype: str, Y: torch.Tensor, c: int, taus) -> list:
    """SPC-ID-ERR (Alg. 6): eps_hat(tau) for each tau, every c-th snapshot."""
    m, n = A.shape
    l = Y.shape[1]
    return ctx.spc_err(A, DTYPE[dtype], m, n, n, Y, l, l, c, taus)
