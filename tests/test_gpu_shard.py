"""The column split of one matrix on the device: P ranks driven from one
process on one GPU (one context each, the sums between them run on the
device by shard.LocalComm), compared with the unsplit path through the C ABI
and with the FP64 oracle.

What must hold (include/lrs.h, column split):
  * the sketch and the subsample are rebuilt exactly (disjoint columns summed
    with zeros), so the C-PWR iterates, the range basis and the row ID --
    r, J and P -- are bit for bit the unsplit path's;
  * with one rank the SVD is bit for bit lrs_svd_k's (the same A-pass, Gram,
    Cholesky and Jacobi);
  * with P ranks the singular values move only by the FP64 rounding of the
    summed Gram (and of B when the slab's A-pass tiles differently): the
    per-value bound of the unsplit path against the oracle holds, and eps
    stays within the 1e-5 relative tolerance of the oracle's;
  * the slabs' rows of V, stacked, reconstruct as the unsplit V does.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import GridSpec

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
C_PIECE = {1: U32, 2: 2.0 ** -16, 3: 2.0 ** -23}
C_TRUNC = {1: 0.0, 2: 16 * U32, 3: 48 * U32}

# the reduced blob recipe (600 x 128^2 FP32, full weighting s = 8 onto 16^2,
# C-PWR on the 2x injection subsample, q = 1, k = 30) with a clear pivot gap
CFG = dict(m=600, N=128, grid=GridSpec((128, 128), (8, 8), "fullweight"),
           gram=GridSpec((128, 128), (2, 2), "inject"), k=30, q=1, rtol=1e-6)
SPIKE = dict(nspikes=30, ratio=0.97, amp0=300.0)
HEAT = synth.WORKLOADS["heat2d_m200_64x64_f64"]


def _torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def gap():
    c = CFG
    A, _ = synth.spiked_blob_field(c["m"], c["N"], 8, 1, s=8, kappa=1e-5, **SPIKE)
    A64 = A.astype(np.float64)
    o = oracle.svd_path(A64, c["grid"], c["k"], q=c["q"], gram_grid=c["gram"], rtol=c["rtol"])
    return A, o


def _unsplit(A_d, dtype, grid, gram, q, k, rtol, prec):
    torch = _torch()
    from paper_2105_01271_gb300 import binding, path
    ctx = binding.load(0, torch.cuda.current_stream())
    m, n = A_d.shape
    b = path.Buffers(m, n, grid.l, k, A_d.device, prec == binding.LRS_PREC_FP64)
    g0, gc = path.power_pass2(ctx, A_d, dtype, grid, q, gram, rtol, prec, b)
    s = path.svd_from_pass(ctx, A_d, dtype, grid, k, q, gc, rtol, prec, b)
    d = path.id_from_pass(ctx, m, grid, k, g0, b)
    torch.cuda.synchronize()
    return ctx, b, s, d


def _split(A_d, dtype, grid, gram, q, k, rtol, prec, world, factor=None):
    torch = _torch()
    from paper_2105_01271_gb300 import binding, shard
    slabs = shard.plan_slabs(grid, gram if q > 0 else None, world)
    local = []
    for sl in slabs:
        ctx = binding.load(0, torch.cuda.current_stream())
        local.append((shard.DeviceOps(ctx), A_d[:, sl.cols[0]:sl.cols[1]].contiguous(), sl))
    cs = shard.ColumnSplit(local, shard.LocalComm(), A_d.shape[0], dtype, grid, gram, q, k, rtol, prec, factor)
    res = cs.step()
    torch.cuda.synchronize()
    return cs, res


def _s_tol(o, A, m, prec):
    QA = np.abs(o["Q"]).T @ np.abs(A)
    c = C_PIECE[prec] + (np.sqrt(m) + 1.0) * U32
    s1 = o["sB"][0]
    sv = o["S"]
    return 6.0 * c * QA.max() + C_TRUNC[prec] * sv + 2.0 ** -44 * s1 ** 2 / sv + 64 * 2.0 ** -53 * s1


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_split_blob_gap(lrs, gap, prec, world):
    torch = _torch()
    from paper_2105_01271_gb300 import binding
    A, o = gap
    c = CFG
    A_d = torch.from_numpy(A).cuda()
    _, b, s, d = _unsplit(A_d, "f32", c["grid"], c["gram"], c["q"], c["k"], c["rtol"], prec)
    cs, res = _split(A_d, "f32", c["grid"], c["gram"], c["q"], c["k"], c["rtol"], prec, world)
    # the exchanged sketch is the unsplit one, bit for bit, on every rank
    for rk in cs.ranks:
        assert torch.equal(rk.Y, b.Y)
    kk = min(c["k"], s.r)
    for x in res:
        assert x.mode == binding.LRS_FACTOR_GRAM
        assert x.r == s.r
        assert torch.equal(x.J, d.J) and torch.equal(x.P, d.P)
        assert x.err_id == d.err_est
    if world == 1:
        x = res[0]
        assert torch.equal(x.S, s.S) and torch.equal(x.U, s.U) and torch.equal(x.V, s.V)
        assert x.err_svd == s.err_est
        return
    A64 = A.astype(np.float64)
    S = res[0].S.cpu().numpy()
    tol = _s_tol(o, A64, c["m"], prec)
    assert np.all(np.abs(S - o["S"]) <= tol), np.max(np.abs(S - o["S"]) / tol)
    for x in res[1:]:
        assert torch.equal(x.S, res[0].S) and torch.equal(x.U, res[0].U)
    U = res[0].U.cpu().numpy()
    np.testing.assert_allclose(U.T @ U, np.eye(kk), atol=1e-12)
    V = np.concatenate([x.V.cpu().numpy().astype(np.float64) for x in res], axis=0)
    assert V.shape == (A.shape[1], kk)
    eps_g = oracle.rel_fro_error(A64, U, S, V)
    eps_o = oracle.rel_fro_error(A64, o["U"], o["S"], o["V"])
    assert abs(eps_g / eps_o - 1.0) <= 1e-5, (eps_g, eps_o)
    assert abs(res[0].err_svd / s.err_est - 1.0) <= 1e-6


@pytest.mark.parametrize("world", [2, 4])
def test_split_r_form_on_fp32_b(lrs, gap, world):
    """The R form (what the split falls back to when the summed Gram is not
    positive definite) on FP32 B: the ranks' TSQR factors side by side."""
    torch = _torch()
    from paper_2105_01271_gb300 import binding
    A, o = gap
    c = CFG
    A_d = torch.from_numpy(A).cuda()
    _, res = _split(A_d, "f32", c["grid"], c["gram"], c["q"], c["k"], c["rtol"], 2, world,
                    factor=binding.LRS_FACTOR_R)
    A64 = A.astype(np.float64)
    x = res[0]
    assert x.mode == binding.LRS_FACTOR_R and x.r == o["r"]
    U, S = x.U.cpu().numpy(), x.S.cpu().numpy()
    V = np.concatenate([y.V.cpu().numpy().astype(np.float64) for y in res], axis=0)
    # FP32 Householder TSQR of B^T (backward error ~ r u32 ||B|| per level,
    # a few levels): 8 r u32 s_1 on top of the products' bound
    tol = _s_tol(o, A64, c["m"], 2) + 8 * o["r"] * U32 * o["sB"][0]
    assert np.all(np.abs(S - o["S"]) <= tol), np.max(np.abs(S - o["S"]) / tol)
    eps_g = oracle.rel_fro_error(A64, U, S, V)
    eps_o = oracle.rel_fro_error(A64, o["U"], o["S"], o["V"])
    assert abs(eps_g / eps_o - 1.0) <= 1e-5, (eps_g, eps_o)


@pytest.mark.parametrize("world", [1, 2, 4])
def test_split_fp64_heat(lrs, world):
    """FP64 data (q = 0, the range finder on every rank; the R form of B):
    the FP64 path's bar against the oracle."""
    torch = _torch()
    A = synth.make_workload(HEAT)
    o = oracle.svd_path(A, HEAT.grid, HEAT.k, q=0, rtol=1e-14)
    d = oracle.id_path(A, HEAT.grid, HEAT.k)
    A_d = torch.from_numpy(A).cuda()
    _, b, s, dd = _unsplit(A_d, "f64", HEAT.grid, None, 0, HEAT.k, 1e-14, 0)
    _, res = _split(A_d, "f64", HEAT.grid, None, 0, HEAT.k, 1e-14, 0, world)
    for x in res:
        assert x.r == s.r
        assert torch.equal(x.J, dd.J) and torch.equal(x.P, dd.P)
        assert np.array_equal(x.J.cpu().numpy(), d["J"])
        S = x.S.cpu().numpy()
        assert np.max(np.abs(S - o["S"])) <= 1e-12 * o["S"][0]
    V = np.concatenate([y.V.cpu().numpy() for y in res], axis=0)
    eps_g = oracle.rel_fro_error(A, res[0].U.cpu().numpy(), res[0].S.cpu().numpy(), V)
    eps_o = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    assert abs(eps_g - eps_o) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_touch_and_power_pass_from_equal_power_pass2(lrs, gap, prec):
    """lrs_touch + lrs_power_pass_from (W also through a wider buffer, row
    stride > |I|) give lrs_power_pass2's outputs bit for bit."""
    torch = _torch()
    from paper_2105_01271_gb300 import binding as bd
    A, _ = gap
    c = CFG
    A_d = torch.from_numpy(A).cuda()
    m, n, l, nI = A.shape[0], A.shape[1], c["grid"].l, c["gram"].l
    g, gg = bd.grid_of(c["grid"]), bd.grid_of(c["gram"])
    f64 = dict(dtype=torch.float64, device="cuda")
    Y, G0, G, Y2, G02, G2 = (torch.full((m, l), np.nan, **f64) for _ in range(6))
    g0, gc = lrs.power_pass2(A_d, bd.LRS_F32, m, n, g, gg, c["q"], c["rtol"], prec, Y, l, G0, l, G, l)
    wdt = torch.float32 if prec >= bd.LRS_PREC_SPLIT_BF16 else torch.float64
    for ldw in (nI, nI + 40):
        Wb = torch.full((m, ldw), np.nan, dtype=wdt, device="cuda")
        lrs.touch(A_d, bd.LRS_F32, m, n, g, gg, prec, Y2, l, Wb, ldw)
        assert torch.equal(Y2, Y)
        idx = torch.from_numpy(_sub_index(c["gram"])).cuda()
        assert torch.equal(Wb[:, :nI].double(), A_d[:, idx].double())
        g02, gc2 = lrs.power_pass_from(Y2, l, Wb, ldw, m, l, nI, c["q"], c["rtol"], prec, G02, l, G2, l)
        torch.cuda.synchronize()
        assert (g02, gc2) == (g0, gc)
        assert torch.equal(G02[:, :g0], G0[:, :g0]) and torch.equal(G2[:, :gc], G[:, :gc])


def _sub_index(gram):
    # injection points of a 2-D grid, x fastest: (s y_c + s/2) N_x + s x_c + s/2
    sx, sy = gram.s
    Nx, Ny = gram.N
    xs = sx * np.arange(Nx // sx) + sx // 2
    ys = sy * np.arange(Ny // sy) + sy // 2
    return (ys[:, None] * Nx + xs[None, :]).ravel()


def test_split_entry_points_validate(lrs):
    torch = _torch()
    from paper_2105_01271_gb300 import binding as bd
    B = torch.zeros((8, 64), dtype=torch.float64, device="cuda")
    F = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(bd.LrsError, match="Gram form"):          # FP64 B has no Gram form
        lrs.slab_factor(B, 8, 64, bd.LRS_PREC_FP64, bd.LRS_FACTOR_GRAM, F, 8)
    with pytest.raises(bd.LrsError, match="n=4 >= r=8"):
        lrs.slab_factor(B, 8, 4, bd.LRS_PREC_FP64, bd.LRS_FACTOR_R, F, 8)
    with pytest.raises(bd.LrsError, match="mode"):
        lrs.slab_factor(B, 8, 64, bd.LRS_PREC_FP64, 7, F, 8)
    Q = torch.zeros((20, 8), dtype=torch.float64, device="cuda")
    U = torch.zeros((20, 4), dtype=torch.float64, device="cuda")
    S = torch.zeros((4,), dtype=torch.float64, device="cuda")
    V = torch.zeros((64, 4), dtype=torch.float32, device="cuda")
    f2 = torch.ones((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(bd.LrsError, match="nf == r"):
        lrs.svd_from_factor(F, 8, 16, bd.LRS_FACTOR_GRAM, Q, 8, 20, 8, 4, bd.LRS_PREC_FP32, B, 64, f2, U, 4, S, V, 4)
    with pytest.raises(bd.LrsError, match="nf=4 < r=8"):
        lrs.svd_from_factor(F, 8, 4, bd.LRS_FACTOR_R, Q, 8, 20, 8, 4, bd.LRS_PREC_FP64, B, 64, f2, U, 4, S, V, 4)
    with pytest.raises(bd.LrsError, match="strides"):
        lrs.touch(torch.zeros((4, 64), device="cuda"), bd.LRS_F32, 4, 64,
                  bd.make_grid((8, 8), (2, 2), "inject"), bd.make_grid((8, 8), (4, 4), "inject"),
                  bd.LRS_PREC_FP32, torch.zeros((4, 16), dtype=torch.float64, device="cuda"), 16,
                  torch.zeros((4, 4), dtype=torch.float64, device="cuda"), 2)
