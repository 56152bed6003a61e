"""Batching form (many independent matrices through lrs_batch_run).

The executor runs the single-matrix call sequence per item on several
streams, so every output must be bit-identical to running the items one at
a time; two items are also checked against the FP64 oracle.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from synth import GridSpec

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _specs():
    return synth.batch_specs(count=10, seed=11, grids=(32, 64), m_range=(50, 300), k_range=(5, 24))


@pytest.fixture(scope="module")
def batch():
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    specs = _specs()
    mats = [synth.make_batch_matrix(sp) for sp in specs]
    dev = [torch.from_numpy(a).cuda() for a in mats]
    return specs, mats, dev


def _items(specs, dev, prec=2):
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    items = (b.lrs_batch_item * len(specs))()
    outs = []
    for it, sp, A in zip(items, specs, dev):
        k = sp.k
        U = torch.full((sp.m, k), np.nan, dtype=torch.float64, device="cuda")
        S = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
        V = torch.full((sp.n, k), np.nan, dtype=torch.float32, device="cuda")
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


def test_batch_matches_one_by_one_and_across_stream_counts(batch):
    from paper_2105_01271_gb300 import binding as b
    from paper_2105_01271_gb300 import path
    specs, mats, dev = batch
    items1, outs1 = _items(specs, dev)
    b.run_batch(items1, n_streams=1)
    items4, outs4 = _items(specs, dev)
    b.run_batch(items4, n_streams=4)
    h1, h4 = _host(outs1), _host(outs4)
    for i, sp in enumerate(specs):
        assert items1[i].status in (b.LRS_OK, b.LRS_ERANK)
        assert items1[i].r == items4[i].r and items1[i].err_svd == items4[i].err_svd
        assert items1[i].err_id == items4[i].err_id
        for a, c in zip(h1[i], h4[i]):
            assert np.array_equal(a, c, equal_nan=True)
    # the same item through the single-matrix path, one call after another
    ctx = b.load(0)
    for i in (0, 3, 7):
        sp = specs[i]
        g = GridSpec((sp.N, sp.N), (sp.s, sp.s), "fullweight")
        s = path.svd_path(ctx, dev[i], "f32", g, sp.k, q=0, rtol=1e-6, prec=2)
        d = path.id_path(ctx, dev[i], "f32", g, sp.k, q=0, rtol=1e-6, prec=2)
        kk = min(sp.k, s.r)
        assert s.r == items1[i].r
        assert np.array_equal(s.S.cpu().numpy(), h1[i][1][:kk])
        assert np.array_equal(s.U.cpu().numpy(), h1[i][0][:, :kk])
        assert np.array_equal(d.J.cpu().numpy(), h1[i][3])
        assert np.array_equal(d.P.cpu().numpy(), h1[i][4])


def test_batch_items_against_the_oracle(batch):
    from paper_2105_01271_gb300 import binding as b
    specs, mats, dev = batch
    items, outs = _items(specs, dev)
    b.run_batch(items, n_streams=3)
    h = _host(outs)
    for i in (1, 5):
        sp = specs[i]
        A = mats[i].astype(np.float64)
        g = GridSpec((sp.N, sp.N), (sp.s, sp.s), "fullweight")
        o = oracle.svd_path(A, g, sp.k, q=0, rtol=1e-6)
        assert items[i].r == o["r"]
        kk = min(sp.k, o["r"])
        U, S, V = h[i][0][:, :kk], h[i][1][:kk], h[i][2][:, :kk].astype(np.float64)
        eps_g = oracle.rel_fro_error(A, U, S, V)
        eps_o = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
        # FP32 data, split-BF16 A-pass.  eps is ~5e-5 for these heat items, below
        # the 1e-4 where the 1e-5 relative tolerance applies; it is held to the
        # product error bound instead: E = B_gpu - B, ||E||_F <= c || |Q|^T |A| ||_F
        # (c = 3 * 2^-16 + (m + 2) u32), |eps_g^2 - eps_o^2| <= (2 ||E|| eps_o ||A|| + ||E||^2) / ||A||^2
        nA = np.linalg.norm(A)
        c = 3 * 2.0 ** -16 + (sp.m + 2) * 2.0 ** -24
        e_b = c * np.linalg.norm(np.abs(o["Q"]).T @ np.abs(A))
        if eps_o >= 1e-4:
            assert abs(eps_g / eps_o - 1.0) <= 1e-5, (eps_g, eps_o)
        assert abs(eps_g ** 2 - eps_o ** 2) <= (2 * e_b * eps_o * nA + e_b ** 2) / nA ** 2, (eps_g, eps_o)
        d = oracle.id_path(A, g, sp.k, q=0, rtol=1e-6)
        gaps = []
        oracle.row_id(d["G"], sp.k, gaps)
        npre = 0
        for gp in gaps:
            if gp <= 1e-10:
                break
            npre += 1
        # q = 0: the ID runs the FP64 CPQR on the FP64 sketch, and every
        # margin of these items is far above its rounding: all k pivots match
        assert npre == sp.k, (i, npre, min(gaps))
        assert np.array_equal(h[i][3], d["J"])


def test_batch_cpwr_items_against_the_oracle():
    """Batch items with one C-PWR pass (q = 1, 2x injection subsample,
    split-BF16 products) on spiked blob fields, whose every ID pivot has a
    clear margin: J is the oracle's and eps within 1e-5 relative."""
    torch = _torch()
    from paper_2105_01271_gb300 import binding as b
    cases = [(300, 64, 4, 12), (420, 64, 8, 10), (250, 128, 8, 16)]
    items = (b.lrs_batch_item * len(cases))()
    outs, mats = [], []
    for it, (m, N, s, k) in zip(items, cases):
        A, _ = synth.spiked_blob_field(m, N, 6, 40 + N, k, s, ratio=0.97, amp0=300.0)
        Ad = torch.from_numpy(A).cuda()
        mats.append((A, Ad))
        U = torch.empty((m, k), dtype=torch.float64, device="cuda")
        S = torch.empty((k,), dtype=torch.float64, device="cuda")
        V = torch.empty((N * N, k), dtype=torch.float32, device="cuda")
        J = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        P = torch.empty((m, k), dtype=torch.float64, device="cuda")
        it.A, it.dtype, it.m, it.lda = Ad.data_ptr(), b.LRS_F32, m, N * N
        it.sketch = b.make_grid((N, N), (s, s), "fullweight")
        it.gram = b.make_grid((N, N), (2, 2), "inject")
        it.q, it.k, it.prec, it.rtol = 1, k, b.LRS_PREC_SPLIT_BF16, 1e-6
        it.do_svd, it.do_id = 1, 1
        it.U, it.ldu, it.S, it.V, it.ldv = U.data_ptr(), k, S.data_ptr(), V.data_ptr(), k
        it.J, it.P, it.ldp = J.data_ptr(), P.data_ptr(), k
        outs.append((U, S, V, J, P))
    b.run_batch(items, n_streams=2)
    for i, (m, N, s, k) in enumerate(cases):
        assert items[i].status == b.LRS_OK, items[i].error
        A = mats[i][0].astype(np.float64)
        g = GridSpec((N, N), (s, s), "fullweight")
        gi = GridSpec((N, N), (2, 2), "inject")
        o = oracle.svd_path(A, g, k, q=1, gram_grid=gi, rtol=1e-6)
        d = oracle.id_path(A, g, k, q=1, gram_grid=gi, rtol=1e-6)
        U, S, V, J, P = (t.cpu().numpy() for t in outs[i])
        eps_g = oracle.rel_fro_error(A, U, S, V.astype(np.float64))
        eps_o = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
        assert eps_o >= 1e-4 and abs(eps_g / eps_o - 1.0) <= 1e-5, (i, eps_g, eps_o)
        gaps = []
        oracle.row_id(d["G"], k, gaps)
        assert min(gaps) > 1e-2, (i, min(gaps))
        assert np.array_equal(J, d["J"]), i
        assert np.array_equal(P[J], np.eye(k))


def test_autotune_picks_a_candidate(batch):
    from paper_2105_01271_gb300 import binding as b
    specs, mats, dev = batch
    items, _ = _items(specs, dev)
    best, ms = b.autotune_batch(items, candidates=(1, 2, 4))
    assert best in (1, 2, 4) and ms > 0


def test_batch_rejects_bad_arguments():
    from paper_2105_01271_gb300 import binding as b
    lib = b.load_library()
    assert lib.lrs_batch_run(0, None, 3, 2) == b.LRS_EINVAL
    items = (b.lrs_batch_item * 1)()
    assert lib.lrs_batch_run(0, ctypes.cast(items, ctypes.c_void_p), 1, 0) == b.LRS_EINVAL
