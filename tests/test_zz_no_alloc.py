"""lrs_id_k_static: the row ID for callers that must not allocate device memory
while they run (a real-time loop with no time for cudaMalloc, or a host
framework that owns every device allocation).  Its scratch is one device array of the
library, so it must give the same skeleton and coefficients as lrs_id_k, call
after call, whatever the previous call left in that array.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


def _run(lrs, Y, k, static):
    import torch
    m, l = Y.shape
    J = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    P = torch.full((m, k), np.nan, dtype=torch.float64, device="cuda")
    fn = lrs.id_k_static if static else lrs.id_k
    err, st = fn(_dev(Y), m, l, l, k, J, P, k)
    return _np(J), _np(P), err


def test_static_matches_allocating_entry_point_twice(lrs):
    # two different inputs in a row: the second call must not depend on what
    # the first left in the shared scratch
    cases = [(synth.pivot_gap_matrix(300, 200, seed=11), 40),
             (synth.pivot_gap_matrix(180, 260, seed=12), 25)]
    for Y, k in cases:
        Js, Ps, es = _run(lrs, Y, k, static=True)
        Ja, Pa, ea = _run(lrs, Y, k, static=False)
        assert np.array_equal(Js, Ja)
        assert np.array_equal(Ps[Js], np.eye(k))
        np.testing.assert_allclose(Ps, Pa, rtol=1e-9, atol=1e-11)
        assert abs(es - ea) <= 1e-10 * max(ea, 1e-16) + 1e-14
        # and both agree with the oracle's skeleton on these gap inputs
        Jo, Po, eo = oracle.row_id(Y, k)
        assert np.array_equal(Js, Jo)


def test_static_row_slab_route(lrs):
    """Fewer than 128 snapshots: the row ID takes the row-slab pivoted QR (not
    the column-owner one), whose scratch the static array must hold as well."""
    Y = synth.pivot_gap_matrix(100, 64, seed=13)
    k = 20
    for _ in range(2):
        Js, Ps, es = _run(lrs, Y, k, static=True)
        Ja, Pa, ea = _run(lrs, Y, k, static=False)
        assert np.array_equal(Js, Ja)
        assert np.array_equal(Ps[Js], np.eye(k))
        np.testing.assert_allclose(Ps, Pa, rtol=1e-9, atol=1e-11)
        assert abs(es - ea) <= 1e-10 * max(ea, 1e-16) + 1e-14
    Jo, Po, eo = oracle.row_id(Y, k)
    assert np.array_equal(Js, Jo)


def test_static_blob_sketch_size(lrs):
    """The row ID at the blob workload's sketch size (2000 x 1024, k = 50) fits
    the static scratch and matches the allocating entry point."""
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((2000, 1024)) * (0.97 ** np.arange(2000))[:, None]
    Js, Ps, es = _run(lrs, Y, 50, static=True)
    Ja, Pa, ea = _run(lrs, Y, 50, static=False)
    assert np.array_equal(Js, Ja)
    np.testing.assert_allclose(Ps, Pa, rtol=1e-9, atol=1e-11)


def test_static_rejects_oversize_before_any_launch(lrs):
    from paper_2105_01271_gb300.binding import LRS_EINVAL, LrsError
    import torch
    tiny = torch.zeros((1,), dtype=torch.float64, device="cuda")
    J = torch.zeros((8,), dtype=torch.int32, device="cuda")
    with pytest.raises(LrsError) as e:
        lrs.id_k_static(tiny, 4000, 2000, 2000, 8, J, tiny, 8)   # ~64 MB of scratch > 32 MiB
    assert e.value.status == LRS_EINVAL
    assert "static scratch holds" in str(e.value)
