"""Full-size check of the headline workload in the configuration bench.py times:
the 2000 x 512^2 FP32 blob field, full weighting s = 16 onto 32^2 (l = 1024),
one C-PWR pass on the 4x injection subsample, k = 50, split-BF16 products.

The oracle cannot decompose the 2.1 GB matrix in seconds, so this test checks
  * outputs the oracle computes one by one: whole rows of the sketch
    Y = A_f D (paper Sec. 2) for sampled snapshots, element by element;
  * properties that hold at any size: U orthonormal; S positive and
    non-increasing; V = A_f^T U S^-1 on sampled dofs within the product error
    bound; the SVD error estimate is a lower bound of the true error of
    U S V^T (the part of A_f outside range(Q) is the difference) and close to
    it; the row ID has k distinct skeleton snapshots with P(J,:) = I exactly.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def blob_full():
    w = synth.WORKLOADS["blob2d_m2000_512x512_f32"]
    return w, synth.make_workload(w)


def test_blob_full_size(lrs, blob_full):
    import torch
    from paper_2105_01271_gb300 import binding, path
    w, A = blob_full
    m, n, k = w.m, w.n, w.k
    Ad = torch.from_numpy(A).cuda()
    prec = binding.LRS_PREC_SPLIT_BF16
    bufs = path.Buffers(m, n, w.grid.l, k, Ad.device, False)
    res = path.svd_path(lrs, Ad, "f32", w.grid, k, q=w.q, gram=w.gram, rtol=1e-6, prec=prec, bufs=bufs)
    ids = path.id_path(lrs, Ad, "f32", w.grid, k, q=w.q, gram=w.gram, rtol=1e-6, prec=prec, bufs=bufs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)

    # sketch rows, element by element (FP64 sums of exact stencil products)
    rows = np.sort(rng.choice(m, 8, replace=False))
    Yg = bufs.Y.cpu().numpy()[rows]
    Yo = oracle.sketch(A[rows], w.grid)
    bound = 27 * U64 * oracle.sketch(np.abs(A[rows]).astype(np.float64), w.grid) + 1e-300
    assert np.all(np.abs(Yg - Yo) <= bound)

    # U orthonormal (Q to ~1e-13, U_B from the FP32 Jacobi), S ordered
    r = res.r
    U, S = res.U.cpu().numpy(), res.S.cpu().numpy()
    V = res.V.cpu().numpy().astype(np.float64)
    assert U.shape == (m, k) and 0 < k <= r
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-5)
    assert np.all(S > 0) and np.all(np.diff(S) <= 0)

    # V = A_f^T U S^-1 on sampled dofs.  B = Q^T A_f carries the split-BF16
    # product error c |Q|^T |A_f| (c = 3 * 2^-16 + (m + 2) u32), V = B^T U_B S^-1
    # with U_B = Q^T U; V is stored in FP32.
    Q = bufs.G.cpu().numpy()[:, :r]
    UB = Q.T @ U
    cols = np.sort(rng.choice(n, 256, replace=False))
    Ac = A[:, cols].astype(np.float64)
    Vref = (Ac.T @ U) / S
    c = 3 * 2.0 ** -16 + (m + 2) * U32
    tol = c * ((np.abs(Q).T @ np.abs(Ac)).T @ np.abs(UB)) / S + 2.0 ** -23 * np.abs(Vref) + 1e-30
    assert np.all(np.abs(V[cols] - Vref) <= tol)

    # the error estimate (tail of the singular values of B) against the true
    # relative error of U S V^T: a lower bound up to rounding, and close
    e_true = oracle.rel_fro_error(A, U, S, V)
    e_est = res.err_est
    assert 0.0 < e_est <= e_true * (1.0 + 1e-4)
    assert e_true <= 1.05 * e_est

    # row ID: k distinct skeleton snapshots, P(J,:) = I exactly
    J, P = ids.J.cpu().numpy(), ids.P.cpu().numpy()
    assert J.shape == (k,) and len(set(J.tolist())) == k
    assert np.all((J >= 0) & (J < m))
    assert np.array_equal(P[J], np.eye(k))
    assert np.all(np.isfinite(P)) and 0.0 < ids.err_est < 1.0
