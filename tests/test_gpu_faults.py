"""Failure handling without a GPU fault.

* A workspace limit turns the allocation a call needs into LRS_ENOMEM before
  any launch; without the limit the same call succeeds on the same context.
* A grid-barrier wait that nothing releases (one block of a two-block
  cooperative launch never arrives) runs out after a bounded number of polls
  into LRS_ETIMEOUT; the context and the device keep working.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _fresh_context():
    from paper_2105_01271_gb300 import binding
    return binding.Context(0)


def _rank12():
    import torch
    A, _ = synth.low_rank_matrix(90, 700, 12, seed=4, decay=0.6)
    return torch.from_numpy(A).cuda()


def test_workspace_limit_gives_enomem_then_recovers():
    import torch
    from paper_2105_01271_gb300.binding import LRS_ENOMEM, LrsError
    ctx = _fresh_context()
    G = _rank12()
    Q = torch.zeros((90, 90), dtype=torch.float64, device="cuda")
    ctx.set_workspace_limit(4096)
    l0 = ctx.launches
    with pytest.raises(LrsError) as e:
        ctx.range_find(G, 90, 700, 700, 1e-12, Q, 90)
    assert e.value.status == LRS_ENOMEM
    assert ctx.launches == l0                      # refused before any launch
    assert not torch.any(Q != 0)
    ctx.set_workspace_limit(0)
    assert ctx.range_find(G, 90, 700, 700, 1e-12, Q, 90) == 12


def test_barrier_timeout_status_and_recovery():
    import torch
    from paper_2105_01271_gb300.binding import LRS_ETIMEOUT
    ctx = _fresh_context()
    assert ctx.selftest_barrier_timeout(200000) == LRS_ETIMEOUT
    assert "gave up" in ctx.lib.lrs_last_error(ctx.h).decode()
    # the context, its stream and the device keep working
    G = _rank12()
    Q = torch.zeros((90, 90), dtype=torch.float64, device="cuda")
    assert ctx.range_find(G, 90, 700, 700, 1e-12, Q, 90) == 12
    Qn = Q.cpu().numpy()[:, :12]
    np.testing.assert_allclose(Qn.T @ Qn, np.eye(12), atol=1e-12)
