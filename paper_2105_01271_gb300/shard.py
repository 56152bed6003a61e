"""Column split of one matrix over several devices: data parallelism over
slabs of A_f's columns (the per-device steps of include/lrs.h's column
split, the slab plan and the two exchanges).

The sketch A_f D and the subsample A_f(:, I) (Sec. 2, Alg. 7) act on each
coarse cell's own fine points, and Alg. 2's B = Q^T A_f and B B^T are sums
over column slabs.  A rank that holds the columns of whole coarse cells -- a
range of the slowest grid axis whose ends are multiples of both grids'
factors on that axis -- therefore reads only its own columns.  One
decomposition is

  touch (the slab's sketch and subsample columns) -> [sum Y, W]
  -> power_pass_from (C-PWR, the same on every rank) -> range_find
  -> apass_slab (B_p = Q^T A_p, ||A_p||_F^2) -> slab_factor (F_p)
  -> [sum F, fro2] -> svd_from_factor (U, S; V_p = the slab's rows of V)
  ;  id_k on the C-PWR iterate (J, P, the same on every rank)

The exchanges are sums: the ranks' columns of Y and W are disjoint (each
rank zero-fills the others'), so their sum is exact; the r x r Grams add up
to B B^T (LRS_FACTOR_GRAM), or the ranks' R^T factors side by side form an
r x (P r) matrix with B B^T as its Gram (LRS_FACTOR_R, for FP64 B or a Gram
that is not positive definite in FP64).

One process may drive several ranks ("local ranks": several contexts, e.g.
on one device); a Comm sums over the local ranks and then over the
processes.  ``ops`` is the object that runs the steps: ``DeviceOps`` (the C
ABI) for the product; any object with the same methods serves (a host
implementation for tests of the orchestration).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import torch

from .binding import (DTYPE, LRS_ERANK, LRS_FACTOR_GRAM, LRS_FACTOR_R, LRS_PREC_FP64, LRS_PREC_SPLIT_BF16,
                      Context, grid_of)


# ---------------------------------------------------------------------------
# slab plan
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Slab:
    """Rank `rank` of `world`: fine indices [z0, z1) of the slowest axis."""
    rank: int
    world: int
    z0: int
    z1: int
    cols: tuple        # [c0, c1): columns of A_f (dofs)
    coarse: tuple      # [j0, j1): columns of the sketch Y
    sub: tuple         # [i0, i1): columns of the subsample W (empty without a gram grid)
    sketch: object     # the slab's sketch grid (N with the slowest axis cut)
    gram: object       # the slab's gram grid, or None

    @property
    def n(self) -> int:
        return self.cols[1] - self.cols[0]


def _cut(grid, ax: int, length: int):
    N = list(grid.N)
    N[ax] = length
    return replace(grid, N=tuple(N))


def plan_slabs(grid, gram, world: int) -> list:
    """Split the slowest axis of `grid` (and `gram`, same fine grid) into
    `world` contiguous slabs of whole cells of both grids, as equal as the
    cells allow.  grid / gram: objects with N, s, kind (synth.GridSpec)."""
    ax = len(grid.N) - 1
    s = int(grid.s[ax])
    unit = s
    if gram is not None:
        if tuple(gram.N) != tuple(grid.N):
            raise ValueError(f"gram grid {gram.N} differs from the sketch grid {grid.N}")
        sg = int(gram.s[ax])
        unit = s * sg // math.gcd(s, sg)
    if grid.kind == "fullweight" and s < 3:
        raise ValueError(f"full weighting with s={s} on the split axis reaches into the next cell (needs s >= 3)")
    Nax = int(grid.N[ax])
    if Nax % unit:
        raise ValueError(f"axis {ax}: N={Nax} is not a multiple of the common cell {unit}")
    cells = Nax // unit
    if world < 1 or cells < world:
        raise ValueError(f"{cells} cells on the split axis for {world} ranks")
    plane = int(math.prod(grid.N[:ax]))
    cplane = int(math.prod(Nd // sd for Nd, sd in zip(grid.N[:ax], grid.s[:ax])))
    gplane = int(math.prod(Nd // sd for Nd, sd in zip(gram.N[:ax], gram.s[:ax]))) if gram is not None else 0
    base, extra = divmod(cells, world)
    out, start = [], 0
    for p in range(world):
        cnt = base + (1 if p < extra else 0)
        z0, z1 = start * unit, (start + cnt) * unit
        start += cnt
        sub = (z0 // int(gram.s[ax]) * gplane, z1 // int(gram.s[ax]) * gplane) if gram is not None else (0, 0)
        out.append(Slab(p, world, z0, z1, (z0 * plane, z1 * plane), (z0 // s * cplane, z1 // s * cplane), sub,
                        _cut(grid, ax, z1 - z0), _cut(gram, ax, z1 - z0) if gram is not None else None))
    return out


# ---------------------------------------------------------------------------
# exchanges
# ---------------------------------------------------------------------------
class LocalComm:
    """Sums over the local ranks of this process only (one process holds the
    whole world).  The sum runs in rank order, so it is deterministic."""

    def allreduce_sum(self, ts: list):
        if len(ts) == 1:
            return
        acc = ts[0]
        for t in ts[1:]:
            if t.device != acc.device:
                raise ValueError("local ranks of one sum live on different devices")
            acc.add_(t)
        for t in ts[1:]:
            t.copy_(acc)


class DistComm(LocalComm):
    """Sums over the local ranks, then over the processes of a
    torch.distributed group (NCCL between GPUs, gloo on the host)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def allreduce_sum(self, ts: list):
        acc = ts[0]
        for t in ts[1:]:
            acc.add_(t)
        self.dist.all_reduce(acc, group=self.group)
        for t in ts[1:]:
            t.copy_(acc)


# ---------------------------------------------------------------------------
# the steps on a device (C ABI); tensors are row-major views (stride(1) == 1)
# ---------------------------------------------------------------------------
def _ld(t) -> int:
    if t.dim() == 2 and t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("row-major views only")
    return int(t.stride(0)) if t.dim() == 2 else int(t.shape[0])


class DeviceOps:
    """The steps through the C ABI.  The context's stream must be torch's
    current stream on its device: the zero-fills and the sums between the
    steps run there."""

    def __init__(self, ctx: Context):
        self.ctx = ctx

    def touch(self, A, dtype, sketch, gram, prec, Y, W):
        g = grid_of(gram) if gram is not None else None
        self.ctx.touch(A, DTYPE[dtype], A.shape[0], _ld(A), grid_of(sketch), g, prec, Y, _ld(Y),
                       W if gram is not None else None, _ld(W) if gram is not None else 0)

    def power_pass_from(self, Y, W, q, rtol, prec, G0, G):
        m, l = Y.shape
        nI = W.shape[1] if (q > 0 and W is not None) else 0
        return self.ctx.power_pass_from(Y, _ld(Y), W if q > 0 else None, _ld(W) if q > 0 else 0, m, l, nI, q,
                                        rtol, prec, G0, _ld(G0), G, _ld(G))

    def range_find(self, G, gc, rtol, Q):
        return self.ctx.range_find(G, G.shape[0], gc, _ld(G), rtol, Q, _ld(Q))

    def apass_slab(self, A, dtype, Q, r, prec, B, fro2):
        m, n = A.shape
        self.ctx.apass_slab(A, DTYPE[dtype], m, n, _ld(A), Q, _ld(Q), r, prec, B, fro2)

    def slab_factor(self, B, r, prec, mode, F):
        self.ctx.slab_factor(B, r, B.shape[1], prec, mode, F, _ld(F))

    def svd_from_factor(self, F, nf, mode, Q, r, k, prec, B, fro2, U, S, V):
        return self.ctx.svd_from_factor(F, _ld(F), nf, mode, Q, _ld(Q), Q.shape[0], r, k, prec, B, B.shape[1],
                                        fro2, U, _ld(U), S, V, _ld(V))

    def id_k(self, G0, g0c, k, J, P):
        return self.ctx.id_k(G0, G0.shape[0], g0c, _ld(G0), k, J, P, _ld(P))


# ---------------------------------------------------------------------------
# one decomposition over the ranks
# ---------------------------------------------------------------------------
@dataclass
class SplitResult:
    slab: Slab
    U: torch.Tensor          # m x k (the same on every rank)
    S: torch.Tensor          # k
    V: torch.Tensor          # n_p x k: the slab's rows of V
    J: torch.Tensor          # k (the same on every rank)
    P: torch.Tensor          # m x k
    err_svd: float
    err_id: float
    r: int
    mode: int                # LRS_FACTOR_GRAM or LRS_FACTOR_R
    status_svd: int
    status_id: int


class _Rank:
    def __init__(self, ops, A, slab: Slab, m, l, nI, k, rmax, prec, f64v):
        dev = A.device
        f64 = torch.float64
        wdt = torch.float32 if prec >= LRS_PREC_SPLIT_BF16 else f64
        self.ops, self.A, self.slab = ops, A, slab
        self.Y = torch.zeros((m, l), dtype=f64, device=dev)
        self.W = torch.zeros((m, nI), dtype=wdt, device=dev) if nI > 0 else None
        self.G0 = torch.empty((m, l), dtype=f64, device=dev)
        self.G = torch.empty((m, l), dtype=f64, device=dev)
        self.Q = torch.empty((m, rmax), dtype=f64, device=dev)
        self.Bflat = torch.empty((rmax * slab.n,), dtype=f64 if prec == LRS_PREC_FP64 else torch.float32, device=dev)
        self.fro2 = torch.zeros((1,), dtype=f64, device=dev)
        self.U = torch.empty((m, k), dtype=f64, device=dev)
        self.S = torch.empty((k,), dtype=f64, device=dev)
        self.V = torch.empty((slab.n, k), dtype=f64 if f64v else torch.float32, device=dev)
        self.J = torch.empty((k,), dtype=torch.int32, device=dev)
        self.P = torch.empty((m, k), dtype=f64, device=dev)


class ColumnSplit:
    """One matrix split over `world` ranks by columns; this process drives
    the ranks in `local` = [(ops, A_p, slab), ...] (A_p: m x n_p, the slab's
    columns of A_f, on the rank's device).  Buffers are allocated once;
    `step()` runs one SVD + ID and returns a SplitResult per local rank."""

    def __init__(self, local, comm, m: int, dtype: str, grid, gram, q: int, k: int, rtol: float, prec: int,
                 factor: int | None = None):
        if not local:
            raise ValueError("no local ranks")
        self.comm, self.m, self.dtype = comm, m, dtype
        self.grid, self.gram, self.q, self.k, self.rtol, self.prec = grid, gram if q > 0 else None, q, k, rtol, prec
        self.l = int(math.prod(Nd // sd for Nd, sd in zip(grid.N, grid.s)))
        self.nI = int(math.prod(Nd // sd for Nd, sd in zip(gram.N, gram.s))) if self.gram is not None else 0
        self.world = local[0][2].world
        self.factor = factor           # None: the Gram form where it applies, else the R form
        self.rmax = min(m, self.l)
        for _, A, sl in local:
            if A.shape != (m, sl.n):
                raise ValueError(f"rank {sl.rank}: A_p is {tuple(A.shape)}, its slab needs ({m}, {sl.n})")
        self.ranks = [_Rank(ops, A, sl, m, self.l, self.nI, k, self.rmax, prec, prec == LRS_PREC_FP64)
                      for ops, A, sl in local]

    def _factor_and_svd(self, Q, r, mode):
        P = self.world
        Fs, nf = [], r
        for rk in self.ranks:
            if mode == LRS_FACTOR_GRAM:
                F = torch.empty((r, r), dtype=torch.float64, device=rk.A.device)
                rk.ops.slab_factor(rk.B, r, self.prec, mode, F)
            else:
                nf = P * r
                F = torch.zeros((r, nf), dtype=torch.float64, device=rk.A.device)
                p = rk.slab.rank
                rk.ops.slab_factor(rk.B, r, self.prec, mode, F[:, p * r:(p + 1) * r])
            Fs.append(F)
        self.comm.allreduce_sum(Fs)
        out = []
        for rk, F, Qr in zip(self.ranks, Fs, Q):
            out.append(rk.ops.svd_from_factor(F, nf, mode, Qr, r, self.k, self.prec, rk.B, rk.fro2, rk.U, rk.S,
                                              rk.V))
        return out

    def step(self) -> list:
        rs = self.ranks
        # (1) the touch of each slab, into its columns of zero-filled Y, W
        for rk in rs:
            sl = rk.slab
            rk.Y.zero_()
            if rk.W is not None:
                rk.W.zero_()
            rk.ops.touch(rk.A, self.dtype, sl.sketch, sl.gram, self.prec, rk.Y[:, sl.coarse[0]:sl.coarse[1]],
                         rk.W[:, sl.sub[0]:sl.sub[1]] if rk.W is not None else None)
        self.comm.allreduce_sum([rk.Y for rk in rs])
        if self.nI > 0:
            self.comm.allreduce_sum([rk.W for rk in rs])
        # (2)-(3) C-PWR and the range basis, the same on every rank
        Q, r = [], None
        cols = []
        for rk in rs:
            g0c, gc = rk.ops.power_pass_from(rk.Y, rk.W, self.q, self.rtol, self.prec, rk.G0, rk.G)
            cols.append(g0c)
            if self.q > 0:
                rr, Qr = gc, rk.G[:, :gc]
            else:
                rr = rk.ops.range_find(rk.G, gc, self.rtol, rk.Q)
                Qr = rk.Q[:, :rr]
            if r is not None and rr != r:
                raise RuntimeError(f"local ranks disagree on the range rank ({r} vs {rr})")
            r = rr
            Q.append(Qr)
        # (4) the slab's B_p and ||A_p||^2
        for rk, Qr in zip(rs, Q):
            rk.B = rk.Bflat[:r * rk.slab.n].view(r, rk.slab.n)
            rk.ops.apass_slab(rk.A, self.dtype, Qr, r, self.prec, rk.B, rk.fro2)
        self.comm.allreduce_sum([rk.fro2 for rk in rs])
        # (5)-(6) the factor, its sum, and the SVD; a Gram that is not
        # positive definite in FP64 (err_est -1: nothing written) falls back
        # to the R form, on every rank alike (the summed Gram is identical)
        mode = LRS_FACTOR_GRAM if (self.prec != LRS_PREC_FP64 and r <= 128) else LRS_FACTOR_R
        if self.factor is not None:
            mode = self.factor
        sv = self._factor_and_svd(Q, r, mode)
        if mode == LRS_FACTOR_GRAM and any(st == LRS_ERANK and err < 0 for err, st in sv):
            mode = LRS_FACTOR_R
            sv = self._factor_and_svd(Q, r, mode)
        # (7) the row ID of the C-PWR iterate
        out = []
        kk = min(self.k, r)
        for rk, g0c, (err_s, st_s) in zip(rs, cols, sv):
            err_i, st_i = rk.ops.id_k(rk.G0, g0c, self.k, rk.J, rk.P)
            out.append(SplitResult(rk.slab, rk.U[:, :kk], rk.S[:kk], rk.V[:, :kk], rk.J, rk.P, err_s, err_i, r,
                                   mode, st_s, st_i))
        return out
