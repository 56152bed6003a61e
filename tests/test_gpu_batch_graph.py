"""The batch as one CUDA graph (lrs_batch_graph_*): the recorded eager run,
then one graph launch for the whole batch, against lrs_batch_run.

Every kernel of the replay takes the same arguments as the eager calls, and
each host read-back is replaced by the recorded value (guarded on the
device), so a launch must give lrs_batch_run's outputs bit for bit on the
same data, with no item run again; the error estimates, computed on the
device in the replay, agree to rounding.  New data in the same buffers is
decomposed by the launch as lrs_batch_run decomposes it: the check scales
every matrix by 2 (exact in every storage type, so ranks and pivots stay and
no guard fires).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _specs():
    return synth.batch_specs(count=16, seed=23, grids=(32, 64, 128), m_range=(50, 400), k_range=(5, 30))


def _items(specs, dev, precs):
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    items = (b.lrs_batch_item * len(specs))()
    outs = []
    for i, (it, sp, A) in enumerate(zip(items, specs, dev)):
        k = sp.k
        prec = precs[i % len(precs)]
        f64 = prec == b.LRS_PREC_FP64
        U = torch.full((sp.m, k), np.nan, dtype=torch.float64, device="cuda")
        S = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
        V = torch.full((sp.n, k), np.nan, dtype=torch.float64 if f64 else torch.float32, device="cuda")
        J = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        P = torch.full((sp.m, k), np.nan, dtype=torch.float64, device="cuda")
        it.A, it.dtype, it.m, it.lda = A.data_ptr(), b.LRS_F32, sp.m, sp.n
        it.sketch = b.make_grid((sp.N, sp.N), (sp.s, sp.s), "fullweight")
        it.q, it.k, it.prec, it.rtol = 0, k, prec, 1e-6
        it.do_svd, it.do_id = 1, 1
        it.U, it.ldu, it.S, it.V, it.ldv = U.data_ptr(), k, S.data_ptr(), V.data_ptr(), k
        it.J, it.P, it.ldp = J.data_ptr(), P.data_ptr(), k
        outs.append((U, S, V, J, P))
    return items, outs


def _host(outs):
    return [[t.cpu().numpy().copy() for t in o] for o in outs]


def _clear(outs):
    for o in outs:
        for t in o:
            t.fill_(-7)


def _same(items_a, h_a, items_b, h_b, err_rtol=1e-14):
    from paper_2105_01271_gb300 import binding as b
    for i in range(len(items_a)):
        a, c = items_a[i], items_b[i]
        assert a.status == c.status and a.r == c.r, i
        assert a.status in (b.LRS_OK, b.LRS_ERANK)
        assert abs(a.err_svd - c.err_svd) <= err_rtol * abs(c.err_svd) + 1e-300, (i, a.err_svd, c.err_svd)
        assert abs(a.err_id - c.err_id) <= err_rtol * abs(c.err_id) + 1e-300, (i, a.err_id, c.err_id)
        kk = min(c.k, c.r)
        id_written = not np.all(h_b[i][3] == -1)      # an ID that ended LRS_ERANK writes no J, P
        for t, (x, y) in enumerate(zip(h_a[i], h_b[i])):
            if t in (0, 1, 2):            # U, S, V: the first min(k, r) directions are written
                x, y = x[..., :kk], y[..., :kk]
            elif not id_written:
                continue
            assert np.array_equal(x, y, equal_nan=True), (i, t)


@pytest.mark.parametrize("branches", [1, 4])
def test_graph_launch_equals_the_eager_batch(lrs, branches):
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    specs = _specs()
    dev = [torch.from_numpy(synth.make_batch_matrix(sp)).cuda() for sp in specs]
    precs = [b.LRS_PREC_SPLIT_BF16, b.LRS_PREC_FP32, b.LRS_PREC_BF16X3, b.LRS_PREC_FP64]
    ref_items, ref_outs = _items(specs, dev, precs)
    b.run_batch(ref_items, n_streams=2)
    ref = _host(ref_outs)
    items, outs = _items(specs, dev, precs)
    g = b.BatchGraph(items, branches=branches)           # the recorded run writes the results
    _same(items, _host(outs), ref_items, ref)
    for _ in range(2):                                  # two launches in a row
        _clear(outs)
        assert g.launch(items) == 0
        torch.cuda.synchronize()
        _same(items, _host(outs), ref_items, ref)
    # new data in the same buffers (every matrix times 2): the launch decomposes it
    for A in dev:
        A.mul_(2.0)
    ref2_items, ref2_outs = _items(specs, dev, precs)
    b.run_batch(ref2_items, n_streams=2)
    _clear(outs)
    assert g.launch(items) == 0
    torch.cuda.synchronize()
    _same(items, _host(outs), ref2_items, _host(ref2_outs))
    g.close()


def test_graph_validates_its_items(lrs):
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    specs = _specs()[:3]
    dev = [torch.from_numpy(synth.make_batch_matrix(sp)).cuda() for sp in specs]
    items, outs = _items(specs, dev, [b.LRS_PREC_SPLIT_BF16])
    items[1].q = 1
    with pytest.raises(b.LrsError):
        b.BatchGraph(items, branches=2)
    items[1].q = 0
    g = b.BatchGraph(items, branches=2)
    items[2].k = items[2].k - 1                          # not the captured batch
    with pytest.raises(b.LrsError):
        g.launch(items)
    g.close()
