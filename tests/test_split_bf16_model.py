"""Host model of the precision form's dense products (the BF16-piece
products on the tensor cores): checked in numpy without a GPU.

The kernels split every operand value into S BF16 pieces, x = x_0 + ... +
x_{S-1} + (rest), each piece the round-to-nearest-even BF16 of what the
previous pieces left (an FP32 value directly; an FP64 value through its
round-to-nearest FP32), and sum the piece products x_i a_j with i + j < S in
FP32.  What must hold, per product, for the constants the GPU parity tests
use (c_2 = 3 * 2^-16, c_3 = 6 * 2^-24):

  * every piece is exact in BF16 (its FP32 bits have zero low halves), and the
    residual after S pieces is within 2^-8S |x| (2^-16 for two pieces; for
    three, zero for an FP32 value and within 2^-24 |x| for an FP64 one);
  * the kept piece products differ from the exact product x a by at most
    c_S |x| |a|, for FP32 and FP64 operands, at random values across
    exponents and at the values that stress the rounding (ties, the largest
    significands, powers of two).
"""
import math

import numpy as np
import pytest
import torch

F32 = np.float32


def bf16_rne(v):
    """Round FP32 values to BF16 (round to nearest, ties to even) in integer
    arithmetic; returns the BF16 values as FP32."""
    u = np.asarray(v, dtype=F32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(F32)


def split(v, S, from_f64=False):
    """The kernels' split: piece i = BF16(rest), rest -= piece (in the
    operand's precision)."""
    if from_f64:
        r = np.asarray(v, dtype=np.float64).copy()
        out = []
        for _ in range(S):
            p = bf16_rne(r.astype(F32))
            out.append(p)
            r = r - p.astype(np.float64)
        return out
    r = np.asarray(v, dtype=F32).copy()
    out = []
    for _ in range(S):
        p = bf16_rne(r)
        out.append(p)
        r = (r - p).astype(F32)
    return out


def kept_product(xp, ap):
    """sum of x_i a_j over i + j < S, each product exact, summed correctly rounded."""
    S = len(xp)
    n = xp[0].size
    out = np.empty(n)
    for e in range(n):
        terms = [float(xp[i][e]) * float(ap[j][e]) for i in range(S) for j in range(S) if i + j < S]
        out[e] = math.fsum(terms)
    return out


def stress_values(rng, n, f64=False):
    """random values over many binades, plus values at rounding boundaries"""
    dt = np.float64 if f64 else F32
    v = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-40, 41, n))
    special = []
    for e in (-20, -1, 0, 1, 7, 30):
        base = np.ldexp(1.0, e)
        special += [base, -base, base * (2 - 2.0 ** -23), base * (1 + 2.0 ** -8),     # exactly a BF16 tie
                    base * (1 + 2.0 ** -8 + 2.0 ** -23), base * (1 + 3 * 2.0 ** -8),  # odd last bit: tie goes up
                    base * (1 + 2.0 ** -16), base * (1 + 2.0 ** -16 + 2.0 ** -23)]
    return np.concatenate([v, np.array(special)]).astype(dt)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    v = stress_values(rng, 20000)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(bf16_rne(v), ref)


@pytest.mark.parametrize("S", [2, 3])
@pytest.mark.parametrize("from_f64", [False, True])
def test_pieces_exact_and_residual_bounded(S, from_f64):
    rng = np.random.default_rng(10 + S + 2 * from_f64)
    v = stress_values(rng, 20000, f64=from_f64)
    pieces = split(v, S, from_f64)
    for p in pieces:
        assert np.all((p.view(np.uint32) & 0xFFFF) == 0)
    x = v.astype(np.float64)
    resid = x - sum(p.astype(np.float64) for p in pieces)
    # FP32 operands: each piece takes >= 8 more significant bits; FP64
    # operands: the FP32 rounding of the rest adds 2^-24 relative per step
    bound = (2.0 ** (-8 * S) if not from_f64 else 2.0 ** (-8 * S) * (1 + 2.0 ** -20)) * np.abs(x)
    assert np.all(np.abs(resid) <= bound)
    if S == 3 and not from_f64:
        # 24 significant bits in three 8-bit pieces (the sign of each piece
        # carries the rounding): an FP32 value is split exactly
        assert np.all(resid == 0.0)


@pytest.mark.parametrize("S,c", [(2, 3 * 2.0 ** -16), (3, 6 * 2.0 ** -24)])
@pytest.mark.parametrize("x_f64", [False, True])
def test_kept_piece_products_within_c_p(S, c, x_f64):
    # X may be FP64 (the FP64 basis Q), A is FP32 data
    rng = np.random.default_rng(100 + S + 3 * x_f64)
    n = 6000
    x = stress_values(rng, n - 48, f64=x_f64)
    a = stress_values(rng, n - 48)
    rng.shuffle(a)
    xp = split(x, S, from_f64=x_f64)
    ap = split(a, S)
    got = kept_product(xp, ap)
    exact = x.astype(np.float64) * a.astype(np.float64)       # exact for FP32 x; within 2^-53 otherwise
    err = np.abs(got - exact)
    mag = np.abs(x.astype(np.float64)) * np.abs(a.astype(np.float64))
    slack = 2.0 ** -52 * mag                                   # the FP64 reference's own rounding
    assert np.all(err <= c * mag + slack), float(np.max((err - slack) / mag))
    # the bound is not loose by orders of magnitude: the worst case uses a
    # good part of it (a dropped term or a residual is ~ c / 3 of |x a|)
    assert float(np.max(err / mag)) > c / 64
