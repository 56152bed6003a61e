"""The column split of one matrix (data parallel over slabs of A_f's
columns) on the host: the slab plan, the locality it relies on, and the
orchestration with its sums over ranks -- in one process (local ranks) and
over world-size-2 gloo process groups -- against the unsplit FP64 oracle.

The per-rank steps come from tests/shard_host_ops.py (the oracle's
routines), so these tests check the split itself: which columns a rank
owns, where its sketch and subsample columns go, that the sums over ranks
rebuild Y, W, B B^T (or its R form) and ||A_f||_F^2, and that V comes back
slab by slab.  The same orchestration drives the device steps in
tests/test_gpu_shard.py.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import GridSpec
from paper_2105_01271_gb300 import shard
from paper_2105_01271_gb300.binding import LRS_FACTOR_GRAM, LRS_FACTOR_R, LRS_PREC_FP32, LRS_PREC_FP64

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from shard_host_ops import HostOps  # noqa: E402

# 2-D, 32 x 32 fine grid (x first), full weighting s = 4 onto 8 x 8, C-PWR
# subsample by 2x injection: cells of lcm(4, 2) = 4 rows, 8 on the split axis
N = 32
GRID = GridSpec(N=(N, N), s=(4, 4), kind="fullweight")
GRAM = GridSpec(N=(N, N), s=(2, 2), kind="inject")


def _field(m=60, nspikes=12, seed=5):
    A, _ = synth.spiked_blob_field(m, N, 3, seed, nspikes=nspikes, s=4, ratio=0.8, amp0=50.0, dtype="f64")
    return A


# ---------------------------------------------------------------------------
# the plan
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("grid,gram,world", [
    (GRID, GRAM, 1), (GRID, GRAM, 2), (GRID, GRAM, 3), (GRID, GRAM, 8), (GRID, None, 5),
    (GridSpec(N=(12, 8, 30), s=(3, 2, 3), kind="fullweight"), GridSpec(N=(12, 8, 30), s=(2, 2, 5), kind="inject"), 2),
    (GridSpec(N=(96,), s=(8,), kind="blockavg"), GridSpec(N=(96,), s=(3,), kind="inject"), 4),
])
def test_plan_slabs_tile_every_index_range(grid, gram, world):
    sl = shard.plan_slabs(grid, gram, world)
    assert [s.rank for s in sl] == list(range(world))
    ax = len(grid.N) - 1
    assert sl[0].z0 == 0 and sl[-1].z1 == grid.N[ax]
    for a, b in zip(sl, sl[1:]):
        assert a.z1 == b.z0 and a.cols[1] == b.cols[0] and a.coarse[1] == b.coarse[0] and a.sub[1] == b.sub[0]
    assert sl[-1].cols[1] == grid.n and sl[-1].coarse[1] == grid.l
    assert sl[-1].sub[1] == (gram.l if gram is not None else 0)
    sizes = [s.z1 - s.z0 for s in sl]
    assert max(sizes) - min(sizes) <= (sizes[0] if world > 1 else 0)     # as equal as whole cells allow
    for s in sl:
        assert s.n == s.sketch.n and s.coarse[1] - s.coarse[0] == s.sketch.l
        if gram is not None:
            assert s.sub[1] - s.sub[0] == s.gram.l


def test_plan_slabs_rejects_what_does_not_split():
    with pytest.raises(ValueError, match="s >= 3"):          # the stencil reaches into the next cell
        shard.plan_slabs(GridSpec(N=(16, 16), s=(2, 2), kind="fullweight"), None, 2)
    with pytest.raises(ValueError, match="multiple"):
        shard.plan_slabs(GridSpec(N=(16, 18), s=(4, 6), kind="inject"), GridSpec(N=(16, 18), s=(2, 4), kind="inject"), 2)
    with pytest.raises(ValueError, match="cells"):
        shard.plan_slabs(GRID, GRAM, 9)
    with pytest.raises(ValueError, match="differs"):
        shard.plan_slabs(GRID, GridSpec(N=(16, 16), s=(2, 2), kind="inject"), 2)


@pytest.mark.parametrize("grid,gram", [
    (GRID, GRAM),
    (GridSpec(N=(12, 8, 30), s=(3, 2, 3), kind="fullweight"), GridSpec(N=(12, 8, 30), s=(2, 2, 5), kind="inject")),
    (GridSpec(N=(12, 8, 30), s=(3, 2, 3), kind="blockavg"), None),
])
def test_a_slab_sketches_its_own_columns(grid, gram):
    # the locality the split relies on: the sketch (and subsample) of a
    # slab's columns are the full sketch's (subsample's) columns of that slab
    rng = np.random.default_rng(3)
    A = rng.standard_normal((7, grid.n))
    Y = oracle.sketch(A, grid)
    W = oracle.subsample(A, gram) if gram is not None else None
    for s in shard.plan_slabs(grid, gram, 2 if gram is not None and len(grid.N) == 3 else 4):
        Ap = A[:, s.cols[0]:s.cols[1]]
        np.testing.assert_allclose(oracle.sketch(Ap, s.sketch), Y[:, s.coarse[0]:s.coarse[1]], rtol=0, atol=1e-15)
        if gram is not None:
            assert np.array_equal(oracle.subsample(Ap, s.gram), W[:, s.sub[0]:s.sub[1]])


def test_full_weighting_with_s2_is_not_slab_local():
    # why plan_slabs needs s >= 3 for full weighting: with s = 2 the stencil
    # of the last coarse row of a slab reads the first fine row of the next
    g = GridSpec(N=(8, 8), s=(2, 2), kind="fullweight")
    half = GridSpec(N=(8, 4), s=(2, 2), kind="fullweight")
    A = np.random.default_rng(4).standard_normal((5, 64))
    Y = oracle.sketch(A, g)
    Yp = oracle.sketch(A[:, :32], half)
    np.testing.assert_allclose(Yp[:, :4], Y[:, :4], rtol=0, atol=1e-15)      # coarse row 0: inside
    assert np.max(np.abs(Yp[:, 4:8] - Y[:, 4:8])) > 1e-3                      # coarse row 1: reads row 4


# ---------------------------------------------------------------------------
# one process, several local ranks
# ---------------------------------------------------------------------------
def _reference(A, k, q, rtol):
    o = oracle.svd_path(A, GRID, k, q=q, gram_grid=GRAM, rtol=rtol)
    d = oracle.id_path(A, GRID, k, q=q, gram_grid=GRAM, rtol=rtol)
    return o, d


def _run_local(A, world, ranks, k, q, rtol, prec):
    slabs = shard.plan_slabs(GRID, GRAM if q > 0 else None, world)
    local = [(HostOps(), torch.from_numpy(np.ascontiguousarray(A[:, slabs[p].cols[0]:slabs[p].cols[1]])), slabs[p])
             for p in ranks]
    cs = shard.ColumnSplit(local, shard.LocalComm(), A.shape[0], "f64", GRID, GRAM, q, k, rtol, prec)
    return cs.step()


def _check(res, o, d, A, tol_s, tol_v):
    k = len(o["S"])
    s1 = o["S"][0]
    for x in res:
        assert x.r == o["r"]
        np.testing.assert_allclose(x.S.numpy(), o["S"], rtol=0, atol=tol_s * s1)
        # U and the slab's rows of V against the oracle's (same sign convention)
        np.testing.assert_allclose(x.U.numpy(), o["U"], rtol=0, atol=tol_v)
        c0, c1 = x.slab.cols
        np.testing.assert_allclose(x.V.numpy().astype(np.float64), o["V"][c0:c1], rtol=0, atol=tol_v)
        assert abs(x.err_svd - o["err_est"]) <= 1e-6 * o["err_est"] + 1e-12
        assert np.array_equal(x.J.numpy(), d["J"])
        np.testing.assert_allclose(x.P.numpy(), d["P"], rtol=0, atol=1e-10)
        assert abs(x.err_id - d["err_est"]) <= 1e-12
    # the slabs' V rows, stacked in rank order, are the whole V
    assert sum(x.V.shape[0] for x in res) == A.shape[1] or len(res) < res[0].slab.world
    assert k == res[0].S.shape[0]


@pytest.mark.parametrize("world", [1, 2, 3])
def test_local_ranks_r_form_match_the_unsplit_oracle(world):
    # FP64 products: B stays FP64 and the R form (the ranks' R^T side by side)
    A = _field()
    k, q, rtol = 10, 1, 1e-10
    o, d = _reference(A, k, q, rtol)
    res = _run_local(A, world, range(world), k, q, rtol, LRS_PREC_FP64)
    assert all(x.mode == LRS_FACTOR_R for x in res)
    _check(res, o, d, A, 1e-12, 1e-9)


@pytest.mark.parametrize("world", [1, 2, 4])
def test_local_ranks_gram_form_match_the_unsplit_oracle(world):
    # FP32 B (as the device stores it) and the summed r x r Gram
    A = _field()
    k, q, rtol = 10, 1, 1e-6
    o, d = _reference(A, k, q, rtol)
    res = _run_local(A, world, range(world), k, q, rtol, LRS_PREC_FP32)
    assert all(x.mode == LRS_FACTOR_GRAM for x in res)
    # B rounded to FP32: singular values to ~u32 of s_1, vectors to ~u32 / gap
    _check(res, o, d, A, 1e-6, 2e-4)


def test_q0_split_takes_the_range_finder():
    A = _field()
    k, rtol = 8, 1e-10
    o = oracle.svd_path(A, GRID, k, q=0, rtol=rtol)
    d = oracle.id_path(A, GRID, k, q=0)
    res = _run_local(A, 2, range(2), k, 0, rtol, LRS_PREC_FP64)
    _check(res, o, d, A, 1e-12, 1e-9)


def test_a_dropped_sum_is_caught():
    # a comm that skips the exchange leaves each rank with its own slab's
    # sketch only: the result must differ from the unsplit one
    class NoComm:
        def allreduce_sum(self, ts):
            pass
    A = _field()
    slabs = shard.plan_slabs(GRID, GRAM, 2)
    local = [(HostOps(), torch.from_numpy(np.ascontiguousarray(A[:, s.cols[0]:s.cols[1]])), s) for s in slabs]
    res = shard.ColumnSplit(local, NoComm(), A.shape[0], "f64", GRID, GRAM, 1, 10, 1e-10, LRS_PREC_FP64).step()
    o, _ = _reference(A, 10, 1, 1e-10)
    assert np.max(np.abs(res[0].S.numpy() - o["S"])) > 1e-3 * o["S"][0]


# ---------------------------------------------------------------------------
# gloo process groups
# ---------------------------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _proc_main(proc, nproc, per_proc, port, out_dir, prec):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=proc, world_size=nproc)
    try:
        from shard_host_ops import HostOps as HO
        A = _field()
        world = nproc * per_proc
        slabs = shard.plan_slabs(GRID, GRAM, world)
        mine = [slabs[proc * per_proc + i] for i in range(per_proc)]
        local = [(HO(), torch.from_numpy(np.ascontiguousarray(A[:, s.cols[0]:s.cols[1]])), s) for s in mine]
        rtol = 1e-10 if prec == LRS_PREC_FP64 else 1e-6
        res = shard.ColumnSplit(local, shard.DistComm(), A.shape[0], "f64", GRID, GRAM, 1, 10, rtol, prec).step()
        for x in res:
            np.savez(os.path.join(out_dir, f"rank{x.slab.rank}.npz"), U=x.U.numpy(), S=x.S.numpy(),
                     V=x.V.numpy().astype(np.float64), J=x.J.numpy(), P=x.P.numpy(),
                     meta=json.dumps({"r": x.r, "mode": x.mode, "err_svd": x.err_svd, "err_id": x.err_id,
                                      "cols": list(x.slab.cols)}))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("per_proc,prec", [(1, LRS_PREC_FP64), (1, LRS_PREC_FP32), (2, LRS_PREC_FP64)])
def test_gloo_world_matches_the_unsplit_oracle(tmp_path, per_proc, prec):
    import torch.multiprocessing as mp
    nproc = 2
    mp.start_processes(_proc_main, args=(nproc, per_proc, _free_port(), str(tmp_path), prec), nprocs=nproc,
                       start_method="spawn", join=True)
    A = _field()
    rtol = 1e-10 if prec == LRS_PREC_FP64 else 1e-6
    o, d = _reference(A, 10, 1, rtol)
    world = nproc * per_proc
    Vs = []
    for p in range(world):
        z = np.load(tmp_path / f"rank{p}.npz")
        meta = json.loads(str(z["meta"]))
        tol_s, tol_v = (1e-12, 1e-9) if prec == LRS_PREC_FP64 else (1e-6, 2e-4)
        assert meta["r"] == o["r"]
        assert meta["mode"] == (LRS_FACTOR_R if prec == LRS_PREC_FP64 else LRS_FACTOR_GRAM)
        np.testing.assert_allclose(z["S"], o["S"], rtol=0, atol=tol_s * o["S"][0])
        np.testing.assert_allclose(z["U"], o["U"], rtol=0, atol=tol_v)
        assert np.array_equal(z["J"], d["J"])
        np.testing.assert_allclose(z["P"], d["P"], rtol=0, atol=1e-10)
        Vs.append(z["V"])
    V = np.concatenate(Vs, axis=0)
    assert V.shape == o["V"].shape
    np.testing.assert_allclose(V, o["V"], rtol=0, atol=1e-9 if prec == LRS_PREC_FP64 else 2e-4)


def test_a_gram_that_is_not_positive_definite_falls_back_to_the_r_form():
    # the device's svd_from_factor answers LRS_ERANK with err_est = -1 when
    # the summed Gram's Cholesky stops early; the split then redoes the
    # factor in the R form on every rank and gets the R form's result
    from paper_2105_01271_gb300.binding import LRS_ERANK

    class GramFails(HostOps):
        calls = []

        def svd_from_factor(self, F, nf, mode, *a):
            GramFails.calls.append(mode)
            if mode == LRS_FACTOR_GRAM:
                return -1.0, LRS_ERANK
            return super().svd_from_factor(F, nf, mode, *a)

    A = _field()
    k, rtol = 10, 1e-6
    slabs = shard.plan_slabs(GRID, GRAM, 2)
    local = [(GramFails(), torch.from_numpy(np.ascontiguousarray(A[:, s.cols[0]:s.cols[1]])), s) for s in slabs]
    res = shard.ColumnSplit(local, shard.LocalComm(), A.shape[0], "f64", GRID, GRAM, 1, k, rtol,
                            LRS_PREC_FP32).step()
    assert GramFails.calls == [LRS_FACTOR_GRAM] * 2 + [LRS_FACTOR_R] * 2
    o, d = _reference(A, k, 1, rtol)
    assert all(x.mode == LRS_FACTOR_R for x in res)
    _check(res, o, d, A, 1e-6, 2e-4)
