"""Full-size check of the headline workload in the configuration bench.py times:
the 2000 x 512^2 FP32 blob field, full weighting s = 16 onto 32^2 (l = 1024),
one C-PWR pass on the 4x injection subsample, k = 50, split-BF16 products.

The oracle takes about a minute per field at this size, so its results are
stored (tests/golden/blob2d_m2000_512x512_f32.json, written by
tests/golden/make_blob2d_full.py from oracle/ and synth/ only).  This test
checks
  * against the stored oracle results: the basis rank r, the relative
    Frobenius error eps of U S V^T within 1e-5 relative, every S_i within the
    per-value bound of tests/test_gpu_path.py, the error estimate within the
    bound propagated from the tail values, and the row ID's error; on the
    clear-pivot-gap variant (synth.spiked_blob_field, 50 spiked snapshots)
    the skeleton J index for index;
  * outputs the oracle computes one by one: whole rows of the sketch
    Y = A_f D (paper Sec. 2) for sampled snapshots, element by element;
  * properties that hold at any size: U orthonormal; S positive and
    non-increasing; V = A_f^T U S^-1 on sampled dofs within the product error
    bound; the SVD error estimate is a lower bound of the true error of
    U S V^T (the part of A_f outside range(Q) is the difference) and close to
    it; the row ID has k distinct skeleton snapshots with P(J,:) = I exactly.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "blob2d_m2000_512x512_f32.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def s_tol(g, m, values):
    """Per-value bound on |s_gpu - s_oracle| for split-BF16 products (see
    tests/test_gpu_path.py): 6 c max(|Q|^T |A_f|) + 16 u32 s_i + 2^-44 s_1^2 / s_i
    + 64 u64 s_1."""
    c = 2.0 ** -16 + (np.sqrt(m) + 1.0) * U32
    s1 = g["sB"][0]
    v = np.asarray(values)
    # + the truncated tensor-core accumulation: 16 MMAs per chunk, < 1 ulp each
    return 6.0 * c * g["absQA_max"] + 16 * U32 * v + 2.0 ** -44 * s1 ** 2 / v + 64 * U64 * s1


def check_svd_against_golden(g, res, A, m, k):
    U, S = res.U.cpu().numpy(), res.S.cpu().numpy()
    V = res.V.cpu().numpy().astype(np.float64)
    assert res.r == g["r"]
    eps = oracle.rel_fro_error(A, U, S, V)
    assert abs(eps / g["eps"] - 1.0) <= 1e-5, (eps, g["eps"])
    tol = s_tol(g, m, g["S"])
    assert np.all(np.abs(S - np.asarray(g["S"])) <= tol), np.max(np.abs(S - g["S"]) / tol)
    tail = np.asarray(g["sB"][k:])
    t = s_tol(g, m, tail)
    b2 = float(np.sum(2.0 * tail * t + t * t) / g["fro2"])
    assert abs(res.err_est ** 2 - g["err_est_svd"] ** 2) <= b2, (res.err_est, g["err_est_svd"], b2)
    return U, S, V, eps


@pytest.fixture(scope="module")
def blob_full():
    w = synth.WORKLOADS["blob2d_m2000_512x512_f32"]
    return w, synth.make_workload(w)


def test_blob_full_size(lrs, blob_full, golden):
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

    # U orthonormal (Q to ~1e-13, U_B from the FP64 Jacobi), S ordered
    r = res.r
    U, S = res.U.cpu().numpy(), res.S.cpu().numpy()
    V = res.V.cpu().numpy().astype(np.float64)
    assert U.shape == (m, k) and 0 < k <= r
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
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

    # against the stored oracle results
    gb = golden["blob"]
    check_svd_against_golden(gb, res, A, m, k)
    # this field has no clear pivot gap (its margins start near 1e-7): the
    # skeleton is not unique at the path's precision, so only its accuracy counts
    assert min(gb["gaps"]) < 1e-2
    e_id = oracle.id_rel_error(A, J, P)
    assert e_id <= gb["id_err"] * (1.0 + 1e-3), (e_id, gb["id_err"])


def test_blob_gap_full_size(lrs, golden):
    """The clear-pivot-gap variant at the full size: J index for index through
    C-PWR with split-BF16 products, and the SVD results against the oracle."""
    import torch
    from paper_2105_01271_gb300 import binding, path
    w = synth.WORKLOADS["blob2d_m2000_512x512_f32"]
    g = golden["spiked"]
    m, n, k = w.m, w.n, w.k
    A, rows = synth.spiked_blob_field(m, w.N, w.params["nblobs"], w.params["seed"], s=w.grid.s[0],
                                      kappa=w.params["kappa"], **g["params"])
    assert np.array_equal(rows, g["spiked_rows"])
    Ad = torch.from_numpy(A).cuda()
    prec = binding.LRS_PREC_SPLIT_BF16
    bufs = path.Buffers(m, n, w.grid.l, k, Ad.device, False)
    res = path.svd_path(lrs, Ad, "f32", w.grid, k, q=w.q, gram=w.gram, rtol=1e-6, prec=prec, bufs=bufs)
    ids = path.id_path(lrs, Ad, "f32", w.grid, k, q=w.q, gram=w.gram, rtol=1e-6, prec=prec, bufs=bufs)
    torch.cuda.synchronize()
    A64 = A.astype(np.float64)
    U, S, V, eps = check_svd_against_golden(g, res, A64, m, k)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
    # every one of the k pivots has a clear margin, so J is the oracle's
    assert min(g["gaps"]) > 1e-2 and len(g["gaps"]) == k
    J, P = ids.J.cpu().numpy(), ids.P.cpu().numpy()
    assert np.array_equal(J, np.asarray(g["J"]))
    assert np.array_equal(P[J], np.eye(k))
    e_id = oracle.id_rel_error(A64, J, P)
    assert abs(e_id / g["id_err"] - 1.0) <= 1e-5, (e_id, g["id_err"])
    assert abs(ids.err_est / g["err_est_id"] - 1.0) <= 1e-5, (ids.err_est, g["err_est_id"])
