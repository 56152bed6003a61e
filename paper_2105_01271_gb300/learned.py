"""Learned sketch proposal (orchestration only; every arithmetic step runs in
liblrs.so through the C ABI).

For a snapshot matrix on an N x N grid the method must pick a sketch before it
knows how much of A_f a sketch captures.  The plain adaptive enlargement tries
the configurations

    CONFIGS = (s, q): (8, 0), (8, 1), (4, 0), (4, 1), (2, 0), (2, 1)   (cheapest first)

in order until the range error of the method's basis meets the tolerance.
The proposal reads the leading 64 diagonal entries of the pivoted R that the
range finder computes for the first configuration's sketch (which either
variant computes anyway), runs the MLP of include/lrs.h on them, and jumps to the predicted configuration, enlarging from there if it
still misses.  `decompose_to_tolerance` runs either variant and reports the
configurations it tried.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .binding import DTYPE, LRS_PREC_SPLIT_BF16, Context, load_library, make_grid

CONFIGS = [(8, 0), (8, 1), (4, 0), (4, 1), (2, 0), (2, 1)]
N_SIGMA, N_IN, N_HID, N_OUT = 64, 67, 128, 6


class Proposal:
    """The MLP's parameters on the device: FP32 master copy, BF16 weights, Adam moments."""

    def __init__(self, ctx: Context, seed: int = 0, device: int = 0):
        self.ctx = ctx
        lib = load_library()
        self.P = int(lib.lrs_mlp_param_count())
        rng = np.random.default_rng(seed)
        p = np.zeros(self.P, dtype=np.float32)
        off = 0
        for (fan_out, fan_in) in ((N_HID, N_IN), (N_HID, N_HID), (N_OUT, N_HID)):
            w = rng.standard_normal((fan_out, fan_in)) * np.sqrt(2.0 / fan_in)
            p[off:off + fan_out * fan_in] = w.ravel()
            off += fan_out * fan_in + fan_out          # biases start at zero
        dev = f"cuda:{device}"
        self.params = torch.from_numpy(p).to(dev)
        self.wbf16 = torch.zeros(self.P, dtype=torch.int16, device=dev)
        self.m1 = torch.zeros(self.P, dtype=torch.float32, device=dev)
        self.m2 = torch.zeros(self.P, dtype=torch.float32, device=dev)
        self.grad = torch.zeros(self.P, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.step = 0
        ctx.mlp_init_bf16(self.params, self.wbf16)

    def loss_grad(self, X: torch.Tensor, y: torch.Tensor):
        self.ctx.mlp_loss_grad(self.params, self.wbf16, X, y, X.shape[0], self.grad, self.loss)
        return self.loss, self.grad

    def train(self, X: np.ndarray, y: np.ndarray, epochs: int = 200, batch: int = 128, lr: float = 2e-3,
              seed: int = 0) -> list:
        """Adam on minibatches (data shuffled per epoch by a seeded permutation); returns
        the mean loss of each epoch."""
        dev = self.params.device
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
        yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.int32)).to(dev)
        rng = np.random.default_rng(seed)
        hist = []
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(len(y))).to(dev)
            tot = 0.0
            nb = 0
            for b0 in range(0, len(y), batch):
                idx = perm[b0:b0 + batch]
                xb = Xd.index_select(0, idx).contiguous()
                yb = yd.index_select(0, idx).contiguous()
                self.loss_grad(xb, yb)
                self.step += 1
                self.ctx.mlp_adam(self.params, self.wbf16, self.grad, self.m1, self.m2, self.step, lr)
                tot += float(self.loss.item())
                nb += 1
            hist.append(tot / max(nb, 1))
        return hist

    def logits(self, X: torch.Tensor) -> torch.Tensor:
        out = torch.empty((X.shape[0], N_OUT), dtype=torch.float32, device=X.device)
        self.ctx.mlp_forward(self.params, self.wbf16, X, X.shape[0], out)
        return out

    def predict(self, X: np.ndarray) -> np.ndarray:
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(self.params.device)
        return self.logits(Xd).argmax(dim=1).cpu().numpy()


@dataclass
class Buffers:
    Y: torch.Tensor
    G: torch.Tensor
    Q: torch.Tensor
    d: torch.Tensor
    x: torch.Tensor


def buffers(m: int, N: int, device) -> Buffers:
    l = (N // 2) ** 2                      # the finest configuration's coarse size
    w = max(l, m)
    f64 = torch.float64
    e = lambda *shape: torch.empty(shape, dtype=f64, device=device)
    return Buffers(e(m, w), e(m, w), e(m, w), e(w), torch.empty((1, N_IN), dtype=torch.float32, device=device))


def basis(ctx: Context, A: torch.Tensor, m: int, N: int, cfg: int, bufs: Buffers, rtol: float = 1e-6,
          diag: bool = False):
    """The method's orthonormal basis for configuration `cfg`: (Q, ldq, r, l).
    With diag (q = 0 only) the range finder also leaves |R_ii| in bufs.d."""
    s, q = CONFIGS[cfg]
    g = make_grid((N, N), (s, s), "fullweight")
    gram = make_grid((N, N), (2, 2), "inject") if q > 0 else None
    l = (N // s) ** 2
    gc = ctx.power_pass(A, DTYPE["f32"], m, N * N, g, gram, q, 1, rtol, LRS_PREC_SPLIT_BF16, bufs.Y, l, bufs.G, l)
    if q > 0:
        return bufs.G, l, gc, l
    ldq = min(m, l)
    if diag:
        r = ctx.range_find_diag(bufs.G, m, gc, l, rtol, bufs.Q, ldq, bufs.d)
    else:
        r = ctx.range_find(bufs.G, m, gc, l, rtol, bufs.Q, ldq)
    return bufs.Q, ldq, r, l


def basis_features(ctx: Context, m: int, N: int, bufs: Buffers, r: int, l: int) -> torch.Tensor:
    """Features of one matrix from the first configuration's range finder
    (|R_ii| in bufs.d, rank r): the feature map of lrs_mlp_features."""
    ctx.mlp_features(bufs.d, min(N_SIGMA, r), r, l, N, m, bufs.x)
    return bufs.x


@dataclass
class ToleranceRun:
    tried: list = field(default_factory=list)     # (configuration, range error)
    accepted: int = -1
    predicted: int = -1
    rank: int = 0
    seconds: float = 0.0


def decompose_to_tolerance(ctx: Context, A: torch.Tensor, m: int, N: int, tol: float, bufs: Buffers,
                           model: Proposal | None = None, start: int | None = None) -> ToleranceRun:
    """Learned start (model given), a fixed start (start given) or the plain
    adaptive enlargement (neither): try configurations from the start upwards
    until the basis captures A to tol, then take the SVD of the accepted basis
    (all r directions)."""
    torch.cuda.synchronize(A.device)
    t0 = time.perf_counter()
    run = ToleranceRun()
    cfg = 0 if start is None else int(start)
    have = False
    if model is not None:
        Q, ldq, r, l = basis(ctx, A, m, N, 0, bufs, diag=True)
        have = True
        x = basis_features(ctx, m, N, bufs, r, l)
        cfg = run.predicted = int(model.logits(x).argmax(dim=1).item())
    while True:
        if not (have and cfg == 0):
            Q, ldq, r, l = basis(ctx, A, m, N, cfg, bufs)
        err = ctx.range_error(A, DTYPE["f32"], m, N * N, N * N, Q, ldq, r) if r > 0 else 1.0
        run.tried.append((cfg, err))
        run.accepted = cfg
        if err <= tol or cfg == len(CONFIGS) - 1:
            break
        cfg += 1
    run.rank = r
    if r > 0:
        dev = A.device
        U = torch.empty((m, r), dtype=torch.float64, device=dev)
        S = torch.empty((r,), dtype=torch.float64, device=dev)
        V = torch.empty((N * N, r), dtype=torch.float32, device=dev)
        ctx.svd_k(A, DTYPE["f32"], m, N * N, N * N, Q, ldq, r, r, LRS_PREC_SPLIT_BF16, U, r, S, V, r)
    torch.cuda.synchronize(A.device)
    run.seconds = time.perf_counter() - t0
    return run
