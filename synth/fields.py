"""Seeded generators for PDE-shaped snapshot matrices A (m snapshots x n dofs).

Layout shared by every consumer: A is row-major, one snapshot per row, and the
dofs of a Cartesian grid are vectorised with x fastest:
    2-D: idx = y*Nx + x            3-D: idx = (z*Ny + y)*Nx + x

Everything is drawn from numpy's PCG64 (``default_rng(seed)``) and computed in
float64, then rounded once to the storage type:
  * f64  -- kept as drawn,
  * f32  -- round-to-nearest-even from float64 (numpy ``astype``),
  * bf16 -- round-to-nearest-even from float64 to 8 significant bits, stored
            as the upper 16 bits of the equal float32 (uint16 bit patterns).

Fields (the paper's data sets are not available, so these stand in for them):
  heat_field       sum of decaying sine modes, the 2-D/3-D heat equation on
                   the unit square/cube with homogeneous Dirichlet walls,
                   interior grid x_p = p/(N+1), p = 1..N.
  blob_field       Gaussian blobs advected with constant velocity on the
                   periodic unit square and spread by diffusion.
  tanh_front_field travelling tanh fronts (slow singular-value decay).
  low_rank_matrix  exact rank-r products with a prescribed spectrum.
  pivot_gap_matrix rows scaled so that column-pivoted QR has a clear gap.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


# ----------------------------------------------------------------------------
# grid description shared by generators, oracle and GPU binding (plain data)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class GridSpec:
    """Fine grid N[0..ndim-1] (x first) with a per-axis coarsening factor s."""
    N: tuple
    s: tuple
    kind: str = "inject"          # "inject" | "fullweight" | "blockavg"

    @property
    def ndim(self) -> int:
        return len(self.N)

    @property
    def n(self) -> int:
        return int(np.prod(self.N))

    @property
    def Nc(self) -> tuple:
        return tuple(Nd // sd for Nd, sd in zip(self.N, self.s))

    @property
    def l(self) -> int:
        return int(np.prod(self.Nc))


# ----------------------------------------------------------------------------
# storage rounding
# ----------------------------------------------------------------------------
def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float64 to bfloat16 (RNE, 8 significant bits); return uint16 bits."""
    x = np.asarray(x, dtype=np.float64)
    mant, expo = np.frexp(x)                      # x = mant * 2**expo, |mant| in [0.5,1)
    r = np.ldexp(np.rint(mant * 256.0), expo - 8)  # rint = round half to even
    f32 = r.astype(np.float32)                     # exact: r has 8 significant bits
    return (f32.view(np.uint32) >> 16).astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    """Exact decode of bfloat16 bit patterns to float64."""
    u = np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def _store(a64: np.ndarray, dtype: str) -> np.ndarray:
    if dtype == "f64":
        return np.ascontiguousarray(a64, dtype=np.float64)
    if dtype == "f32":
        return np.ascontiguousarray(a64.astype(np.float32))
    if dtype == "bf16":
        return np.ascontiguousarray(to_bf16_bits(a64))
    raise ValueError(dtype)


# ----------------------------------------------------------------------------
# heat equation field
# ----------------------------------------------------------------------------
def heat_params(m: int, d: int, K: int, seed: int, nu: float = 0.01):
    """Draws of the heat field: sorted times t ~ U[0,1], coefficients
    c_ij(l) ~ N(0,1)/(1+i+j(+l))^2 and decay rates nu*pi^2*|mode|^2."""
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, 1.0, m))
    modes = np.stack(np.meshgrid(*[np.arange(1, K + 1)] * d, indexing="ij"), -1)
    modes = modes.reshape(-1, d)                        # (K^d, d): (i, j[, l]) with i the x mode
    c = rng.standard_normal(len(modes)) / (1.0 + modes.sum(1)) ** 2
    lam = nu * np.pi ** 2 * (modes ** 2).sum(1)
    return t, modes, c, lam


def heat_field(m: int, N: int, d: int, K: int, seed: int, dtype: str = "f64",
               rows: slice | None = None) -> np.ndarray:
    """u(x,t) = sum_modes c e^{-lam t} prod_axis sin(mode_axis * pi * x_axis).

    Returns rows ``rows`` (default all) of the m x N^d matrix in ``dtype``.
    """
    t, modes, c, lam = heat_params(m, d, K, seed)
    if rows is not None:
        t = t[rows]
    x = np.arange(1, N + 1) / (N + 1.0)
    S = np.sin(np.pi * np.outer(np.arange(1, K + 1), x))        # (K, N): S[i-1, p]
    coef = np.exp(-np.outer(t, lam)) * c                         # (mt, K^d)
    mt = len(t)
    if d == 2:
        C = coef.reshape(mt, K, K)                               # [t, i(x), j(y)]
        # A[t, y, x] = sum_{i,j} C[t,i,j] S[j,y] S[i,x]
        tmp = np.einsum("tij,jy->tiy", C, S)
        A = np.einsum("tiy,ix->tyx", tmp, S).reshape(mt, N * N)
    elif d == 3:
        # separable: three matrix products per chunk of snapshots (BLAS), rounded
        # to the storage type chunk by chunk (the float64 field is never whole);
        # chunks run on a thread pool (numpy and BLAS release the GIL)
        C = coef.reshape(mt, K, K, K)                            # [t, i(x), j(y), l(z)]
        probe = _store(np.zeros((1, 1)), dtype)
        out = np.empty((mt, N * N * N), dtype=probe.dtype)

        def chunk(r0):
            Cb = C[r0:r0 + 4]
            b = len(Cb)
            t1 = (Cb.reshape(b * K * K, K) @ S).reshape(b, K, K, N)                  # [t,i,j,z]
            t2 = np.ascontiguousarray(t1.transpose(0, 1, 3, 2)).reshape(b * K * N, K) @ S
            t2 = t2.reshape(b, K, N, N)                                            # [t,i,z,y]
            t3 = np.ascontiguousarray(t2.transpose(0, 2, 3, 1)).reshape(b * N * N, K) @ S
            out[r0:r0 + b] = _store(t3.reshape(b, N * N * N), dtype)               # [t,(z,y,x)]

        starts = list(range(0, mt, 4))
        if len(starts) > 1 and N ** 3 >= (1 << 18):
            import concurrent.futures as cf
            import os
            with cf.ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
                list(ex.map(chunk, starts))
        else:
            for r0 in starts:
                chunk(r0)
        return out
    else:
        raise ValueError("heat_field supports d = 2 or 3")
    return _store(A, dtype)


# ----------------------------------------------------------------------------
# advected / diffused Gaussian blobs on the periodic unit square
# ----------------------------------------------------------------------------
def blob_params(nblobs: int, seed: int):
    rng = np.random.default_rng(seed)
    c0 = rng.uniform(0.0, 1.0, (nblobs, 2))
    vel = rng.uniform(-1.0, 1.0, (nblobs, 2))
    width = rng.uniform(0.02, 0.1, nblobs)
    amp = rng.standard_normal(nblobs)
    return c0, vel, width, amp


def blob_field(m: int, N: int, nblobs: int, seed: int, kappa: float = 1e-5,
               dtype: str = "f32", rows: slice | None = None) -> np.ndarray:
    """Blob b at time t_i = i/(m-1): centre c0 + v t (mod 1), variance
    w^2 + 2 kappa t, amplitude a w^2/(w^2 + 2 kappa t) (mass kept by diffusion).
    Grid: cell centres (p + 1/2)/N, minimum-image distance per axis."""
    c0, vel, width, amp = blob_params(nblobs, seed)
    t = np.linspace(0.0, 1.0, m) if m > 1 else np.zeros(1)
    if rows is not None:
        t = t[rows]
    xs = (np.arange(N) + 0.5) / N
    out = np.empty((len(t), N * N), dtype=np.float64)
    for r0 in range(0, len(t), 64):
        tb = t[r0:r0 + 64]
        var = width[None, :] ** 2 + 2.0 * kappa * tb[:, None]            # (mt, B)
        cx = (c0[None, :, 0] + vel[None, :, 0] * tb[:, None]) % 1.0
        cy = (c0[None, :, 1] + vel[None, :, 1] * tb[:, None]) % 1.0
        dx = (xs[None, None, :] - cx[:, :, None] + 0.5) % 1.0 - 0.5      # (mt, B, N)
        dy = (xs[None, None, :] - cy[:, :, None] + 0.5) % 1.0 - 0.5
        gx = np.exp(-dx ** 2 / (2.0 * var[:, :, None]))
        gy = np.exp(-dy ** 2 / (2.0 * var[:, :, None]))
        a = amp[None, :] * width[None, :] ** 2 / var                      # (mt, B)
        # A[t, y, x] = sum_b a[t,b] gy[t,b,y] gx[t,b,x]
        blk = np.matmul((gy * a[:, :, None]).transpose(0, 2, 1), gx)     # (mt, N, N)
        out[r0:r0 + len(tb)] = blk.reshape(len(tb), -1)
    return _store(out, dtype)


def spiked_blob_field(m: int, N: int, nblobs: int, seed: int, nspikes: int, s: int,
                      ratio: float = 0.97, amp0: float = 10.0, kappa: float = 1e-5,
                      dtype: str = "f32"):
    """The blob field with a clear pivot gap for the row ID: nspikes snapshots
    (drawn without replacement) each carry one extra Gaussian bump of
    amplitude amp0 * ratio**j (j = 0, 1, ... in draw order).  The bumps sit on
    coarse points of the sketch grid with per-axis factor s, spaced
    Nc // g coarse cells apart (g = ceil(sqrt(nspikes)) per axis, Nc = N / s),
    with standard deviation a quarter of that spacing, so they are nearly
    orthogonal to each other and every one meets the sketch stencil the same
    way.  The spiked rows then dominate the sketch and its C-PWR iterate in
    amplitude order, each pivot ahead of the next by a margin of about
    1 - ratio**3 (the iterate is cubic in the row scale), which the tests
    check rather than assume.  Returns (A, spiked row indices in draw order)."""
    base = blob_field(m, N, nblobs, seed, kappa, "f64")
    rng = np.random.default_rng(seed + 7919)
    rows = rng.choice(m, nspikes, replace=False)
    g = int(np.ceil(np.sqrt(nspikes)))
    Nc = N // s
    step = max(1, Nc // g)
    cells = rng.choice(g * g, nspikes, replace=False)
    sd = step * s / 4.0                              # fine points
    idx = np.arange(N)
    for j in range(nspikes):
        # coarse point (a, b) sits at fine index s * a + s // 2 per axis
        cx = s * ((cells[j] % g) * step) + s // 2
        cy = s * ((cells[j] // g) * step) + s // 2
        dx = (idx - cx + N / 2.0) % N - N / 2.0      # periodic minimum image
        dy = (idx - cy + N / 2.0) % N - N / 2.0
        phi = np.exp(-dy[:, None] ** 2 / (2 * sd * sd)) * np.exp(-dx[None, :] ** 2 / (2 * sd * sd))
        base[rows[j]] += amp0 * ratio ** j * phi.ravel()
    return _store(base, dtype), rows


# ----------------------------------------------------------------------------
# travelling tanh fronts (slow decay)
# ----------------------------------------------------------------------------
def tanh_front_field(m: int, N: int, nfronts: int, seed: int, dtype: str = "f32") -> np.ndarray:
    """Fronts tanh(k (n . x - x0 - c t)) with sharpness k ~ U[10, 200]."""
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, nfronts)
    sharp = rng.uniform(10.0, 200.0, nfronts)
    x0 = rng.uniform(0.2, 0.8, nfronts)
    speed = rng.uniform(-0.5, 0.5, nfronts)
    amp = rng.standard_normal(nfronts)
    t = np.linspace(0.0, 1.0, m)
    xs = (np.arange(N) + 0.5) / N
    X, Yg = np.meshgrid(xs, xs, indexing="xy")           # X[y, x] = x
    out = np.zeros((m, N * N))
    for f in range(nfronts):
        proj = (np.cos(ang[f]) * X + np.sin(ang[f]) * Yg).ravel()
        out += amp[f] * np.tanh(sharp[f] * (proj[None, :] - x0[f] - speed[f] * t[:, None]))
    return _store(out, dtype)


# ----------------------------------------------------------------------------
# matrices with known structure (for pins)
# ----------------------------------------------------------------------------
def low_rank_matrix(m: int, n: int, r: int, seed: int, decay: float = 0.7,
                    dtype: str = "f64"):
    """A = U diag(sigma) V^T with orthonormal U (m x r), V (n x r) and
    sigma_i = decay**i.  Returns (A, sigma)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    sig = decay ** np.arange(r)
    return _store((U * sig) @ V.T, dtype), sig


def pivot_gap_matrix(m: int, n: int, seed: int, ratio: float = 0.8,
                     dtype: str = "f64") -> np.ndarray:
    """Gaussian rows scaled by ratio**perm(i): with row norms spread
    geometrically the pivot choice of a column-pivoted QR of A^T has a clear
    margin at every step (checked by the tests, not assumed)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, n))
    G /= np.linalg.norm(G, axis=1, keepdims=True)
    scale = ratio ** rng.permutation(m)
    return _store(G * scale[:, None], dtype)


# ----------------------------------------------------------------------------
# named workloads (sizes of the paper-shaped configurations)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    field: str
    m: int
    N: int
    d: int
    dtype: str
    grid: GridSpec
    k: int
    q: int
    gram: GridSpec | None = None      # C-PWR column subsample I (injection grid)
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.N ** self.d


def _wl(name, field_, m, N, d, dtype, kind, s, k, q, s_gram=None, **params):
    grid = GridSpec(N=(N,) * d, s=(s,) * d, kind=kind)
    gram = GridSpec(N=(N,) * d, s=(s_gram,) * d, kind="inject") if s_gram else None
    return Workload(name, field_, m, N, d, dtype, grid, k, q, gram, dict(params))


WORKLOADS = {
    # 200 snapshots of the 2-D heat field on 64^2, FP64, 4x injection (l = 256), k = 20
    "heat2d_m200_64x64_f64": _wl("heat2d_m200_64x64_f64", "heat", 200, 64, 2, "f64",
                                 "inject", 4, 20, 0, K=16, seed=0),
    # 2000 blob snapshots on 512^2, FP32, full weighting onto 32^2 (l = 1024), k = 50, q = 1
    "blob2d_m2000_512x512_f32": _wl("blob2d_m2000_512x512_f32", "blob", 2000, 512, 2, "f32",
                                    "fullweight", 16, 50, 1, s_gram=4, nblobs=8, seed=1,
                                    kappa=1e-5),
    # the same blob recipe on 256^2 with the headline's sketch sizes (full weighting s = 8 onto
    # 32^2, l = 1024; C-PWR on the 2x injection subsample, |I| = 16384): a 0.5 GB case for
    # counter captures of the same kernels
    "blob2d_m2000_256x256_f32": _wl("blob2d_m2000_256x256_f32", "blob", 2000, 256, 2, "f32",
                                    "fullweight", 8, 50, 1, s_gram=2, nblobs=8, seed=1,
                                    kappa=1e-5),
    # 500 snapshots of the 3-D heat field on 256^3, BF16, injection onto 8^3 (l = 512), k = 64
    "heat3d_m500_256c_bf16": _wl("heat3d_m500_256c_bf16", "heat", 500, 256, 3, "bf16",
                                 "inject", 32, 64, 0, K=12, seed=2),
}


def make_workload(w: Workload, rows: slice | None = None, seed_offset: int = 0) -> np.ndarray:
    """Materialise (rows of) a workload's A in its storage dtype.  seed_offset
    gives independent matrices of the same recipe (one per rank)."""
    p = w.params
    seed = p["seed"] + seed_offset
    if w.field == "heat":
        return heat_field(w.m, w.N, w.d, p["K"], seed, w.dtype, rows=rows)
    if w.field == "blob":
        return blob_field(w.m, w.N, p["nblobs"], seed, p.get("kappa", 1e-5), w.dtype,
                          rows=rows)
    raise ValueError(w.field)


# ----------------------------------------------------------------------------
# batching form: many matrices of mixed size
# ----------------------------------------------------------------------------
@dataclass
class BatchSpec:
    field: str          # "heat" or "blob"
    m: int
    N: int              # 2-D grid N x N
    s: int              # full-weighting factor per axis (divides N)
    k: int
    seed: int

    @property
    def n(self) -> int:
        return self.N * self.N

    @property
    def l(self) -> int:
        return (self.N // self.s) ** 2


def batch_specs(count: int = 256, seed: int = 3, grids=(32, 64, 128, 256), m_range=(50, 2000),
                k_range=(5, 60), factors=(2, 4, 8)) -> list:
    """Seeded list of independent 2-D FP32 problems: grid N^2 from `grids`,
    m ~ U[m_range], field heat or blob, full-weighting factor from `factors`
    (powers of two, so they divide N), k ~ U[k_range] capped at min(m, l)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice(grids))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        field = "heat" if rng.integers(0, 2) == 0 else "blob"
        sf = int(rng.choice(factors))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        l = (N // sf) ** 2
        out.append(BatchSpec(field, m, N, sf, min(k, m, l), 1000 + i))
    return out


def make_batch_matrix(b: BatchSpec, dtype: str = "f32") -> np.ndarray:
    if b.field == "heat":
        return heat_field(b.m, b.N, 2, 16, b.seed, dtype)
    return blob_field(b.m, b.N, 8, b.seed, 1e-5, dtype)


# ----------------------------------------------------------------------------
# the mixed 2-D set of the learned sketch proposal
# ----------------------------------------------------------------------------
LEARNED_FIELDS = ("heat", "blob", "tanh")


def learned_specs(count: int, seed: int) -> list:
    """Seeded draws of the learned proposal's matrices: 2-D fields on N x N
    grids, N in {32, 64, 128}, m ~ U[64, 512] snapshots, FP32 storage; heat
    (16 modes, 20%), advected blobs (2-16 blobs, 40%), travelling tanh fronts
    (1-4 fronts, sharpness 10-200, 40%)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        out.append(dict(field=LEARNED_FIELDS[int(rng.choice(3, p=[0.2, 0.4, 0.4]))],
                        N=int(rng.choice([32, 64, 128])), m=int(rng.integers(64, 513)),
                        nfronts=int(rng.integers(1, 5)), nblobs=int(rng.integers(2, 17)),
                        seed=int(seed * 100000 + i)))
    return out


def learned_heldout_specs(count: int = 1000, seed: int = 9) -> list:
    """The held-out evaluation set of the learned proposal: 1000 snapshots on
    N x N grids, N in {128, 256, 512} (uniform), the same field mix and
    parameter ranges as learned_specs, seeds disjoint from the training and
    test draws (seed * 100000 + i with seed 9)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        out.append(dict(field=LEARNED_FIELDS[int(rng.choice(3, p=[0.2, 0.4, 0.4]))],
                        N=int(rng.choice([128, 256, 512])), m=1000,
                        nfronts=int(rng.integers(1, 5)), nblobs=int(rng.integers(2, 17)),
                        seed=int(seed * 100000 + i)))
    return out


def learned_matrix(sp: dict) -> np.ndarray:
    if sp["field"] == "heat":
        return heat_field(sp["m"], sp["N"], 2, 16, sp["seed"], "f32")
    if sp["field"] == "blob":
        return blob_field(sp["m"], sp["N"], sp["nblobs"], sp["seed"], 1e-5, "f32")
    return tanh_front_field(sp["m"], sp["N"], sp["nfronts"], sp["seed"], "f32")


def learned_spec_from_meta(row) -> dict:
    """The spec of one stored meta row (field, N, m, fronts, blobs, seed)."""
    f, N, m, nf, nb, seed = (int(v) for v in row)
    return dict(field=LEARNED_FIELDS[f], N=N, m=m, nfronts=nf, nblobs=nb, seed=seed)
