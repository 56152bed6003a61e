"""The Gram B B^T of a wide FP32 B (the small SVD's input, Alg. 2) as an
exact-slice product on the tensor cores, through lrs_slab_factor
(LRS_FACTOR_GRAM), against references that are exact or correctly rounded.

What must hold:
  * integer-valued B whose Gram is exact in FP64 (every slice product and
    every partial sum on the kernel's grids is exact): G bit for bit the
    exact Gram, for one and two column groups, ragged n, zero rows, rows
    scaled by 2^+-100, an unaligned B, and the largest slice values (the
    exact accumulators' worst case);
  * the same at n large enough that a CTA sums several int64 ranges;
  * general FP32 B: every entry within 2^-44 of sum_k |b_ik b_jk| of the
    correctly rounded Gram (math.fsum of the exact FP64 products), the bound
    the double-float Gram it replaces was held to.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _gram(lrs, B, offset=0):
    """G = B B^T on the GPU; offset > 0 places B off a 16-byte boundary."""
    from paper_2105_01271_gb300.binding import LRS_FACTOR_GRAM, LRS_PREC_SPLIT_BF16
    torch = _torch()
    r, n = B.shape
    buf = torch.zeros(offset + B.size, dtype=torch.float32, device="cuda")
    buf[offset:] = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float32).ravel()).cuda()
    Bd = buf[offset:]
    F = torch.empty((r, r), dtype=torch.float64, device="cuda")
    lrs.slab_factor(Bd, r, n, LRS_PREC_SPLIT_BF16, LRS_FACTOR_GRAM, F, r)
    torch.cuda.synchronize()
    return F.cpu().numpy()


def _fsum_gram(B):
    b = B.astype(np.float64)
    r = b.shape[0]
    G = np.empty((r, r))
    for i in range(r):
        for j in range(i, r):
            G[i, j] = G[j, i] = math.fsum(b[i] * b[j])
    return G


def _assert_exact_gram(G, ref):
    assert np.array_equal(G, ref)


def _int_matrix(rng, r, n, bits):
    """Integers below 2^bits in magnitude: a random row, a row at the maximum
    with one sign (the largest slice sums), a zero row."""
    hi = 2 ** bits - 1
    B = rng.integers(-hi, hi + 1, size=(r, n)).astype(np.float64)
    if r > 2:
        B[1] = hi
        B[2] = 0.0
    return B


@pytest.mark.parametrize("r,n", [(1, 1), (5, 37), (17, 1000), (40, 3001), (72, 5000), (96, 4100),
                                 (114, 2999), (128, 1537)])
def test_gram_exact_on_integers(lrs, r, n):
    rng = np.random.default_rng(1000 + r)
    # 20-bit integers: three slices of each value, every level's sums exact;
    # the Gram (< n 2^40 < 2^53) is exact in FP64
    B = _int_matrix(rng, r, n, 20)
    G = _gram(lrs, B.astype(np.float32))
    ref = B @ B.T                       # exact: every partial sum is an integer below 2^53
    _assert_exact_gram(G, ref)


def test_gram_exact_scaled_rows_and_unaligned(lrs):
    rng = np.random.default_rng(7)
    r, n = 24, 2100
    B = _int_matrix(rng, r, n, 16)
    scale = np.ldexp(1.0, rng.integers(-100, 101, size=r)).astype(np.float64)
    Bs = B * scale[:, None]
    ref = B @ B.T * np.outer(scale, scale)          # powers of two: still exact
    G = _gram(lrs, Bs.astype(np.float32), offset=1)
    _assert_exact_gram(G, ref)


@pytest.mark.slow
def test_gram_exact_over_many_ranges(lrs):
    # n large enough that every CTA sums two int64 ranges; 10-bit integers keep
    # the FP64 reference exact (partial sums below 2^41)
    rng = np.random.default_rng(11)
    r, n = 20, 2_700_000
    B = rng.integers(-1023, 1024, size=(r, n)).astype(np.float32)
    G = _gram(lrs, B)
    ref = B.astype(np.float64) @ B.astype(np.float64).T
    _assert_exact_gram(G, ref)


@pytest.mark.parametrize("r,n,kind", [(72, 20000, "gauss"), (114, 9000, "gauss"), (40, 12000, "field"),
                                      (128, 3000, "spread")])
def test_gram_accuracy_fp32(lrs, r, n, kind):
    rng = np.random.default_rng(r + n)
    if kind == "gauss":
        B = rng.standard_normal((r, n)) * np.logspace(0, -4, r)[:, None]
    elif kind == "field":
        # smooth rows of decaying amplitude (the B = Q^T A_f of a field)
        t = np.linspace(0.0, 1.0, n)
        B = np.stack([np.sin(np.pi * (i + 1) * t + rng.uniform()) * 0.7 ** i for i in range(r)])
        B += 1e-6 * rng.standard_normal((r, n))
    else:
        # entries spread over 2^-30..2^30 within each row
        B = rng.standard_normal((r, n)) * np.ldexp(1.0, rng.integers(-30, 31, size=(r, n)))
    B = B.astype(np.float32)
    G = _gram(lrs, B)
    ref = _fsum_gram(B)
    a = np.abs(B.astype(np.float64))
    err = np.abs(G - ref)
    assert np.array_equal(G, G.T)
    if kind != "spread":
        # rows whose entries stay within ~2^20 of their maximum: the
        # double-float Gram's bound, per entry
        bound = a @ a.T
        rel = err / np.where(bound > 0, bound, 1.0)
        assert rel.max() <= 2.0 ** -44, f"max error {rel.max():.3e} of sum |b_i b_j|"
    else:
        # any FP32 rows: the fixed-point bound of the slicing, in units of
        # each row's power-of-two bound m_i (cut 2^-49 m_i below the top)
        m = np.ldexp(1.0, np.frexp(a.max(axis=1))[1])
        A1 = a.sum(axis=1)
        bound = 2.0 ** -46 * (np.outer(m, A1) + np.outer(A1, m) + n * np.outer(m, m))
        assert (err <= bound).all(), f"max error {(err / bound).max():.3e} of the fixed-point bound"
