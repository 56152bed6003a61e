"""Host model of the exact-slice Gram's drain arithmetic (the SVD's Gram of
B, Alg. 2), checked in numpy FP32 without a GPU: the conversions the kernel
makes without a float-to-integer instruction.

  * rint22(v) = bits(v + 1.5 2^23) - bits(1.5 2^23) is round-to-nearest-even
    of v for every FP32 |v| <= 2^22;
  * rint35(v): a = (v 2^-13 + M) - M, rem = fma(a, -2^13, v) (exact), then
    a 2^13 + rint22(rem), is round-to-nearest-even of v for every FP32
    |v| < 2^35 (rem has |rem| <= 2^12 and is v's exact remainder);
  * ll50(v), from v's significand and exponent in integer arithmetic, is
    round-half-up of v 2^50 for every FP32 |v| < 2^12, subnormals included;
  * an accumulator of level L (|a_L| within its stated integer bound, times
    2^-(16 + 8L) as the tensor core holds it) is recovered exactly by the
    drain's scale and rounding, and the five drained terms add into int64
    without overflow over a range of 16384 columns.
"""
from fractions import Fraction

import numpy as np

F32 = np.float32
MAGIC = F32(12582912.0)                   # 1.5 2^23
MAGIC_BITS = 0x4B400000


def rint22(v):
    v = np.asarray(v, dtype=F32)
    return (v + MAGIC).view(np.int32).astype(np.int64) - MAGIC_BITS


def fma32(a, b, c):
    """FP32 fused multiply-add: the exact a b + c rounded once (the product
    of two FP32 values is exact in FP64, and so is this sum when it is an
    exact FP32 remainder, as here)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def rint35(v):
    v = np.asarray(v, dtype=F32)
    a = ((v * F32(1.220703125e-4)) + MAGIC) - MAGIC
    rem = fma32(a, F32(-8192.0), v)
    return rint22(a) * 8192 + rint22(rem)


def ll50(v):
    """round-half-up of v 2^50 from v's bits (v = m 2^(E - 150))."""
    out = []
    for bits in np.asarray(v, dtype=F32).view(np.uint32).tolist():
        E = (bits >> 23) & 0xFF
        m = (bits & 0x7FFFFF) | (0x800000 if E else 0)
        sh = (E if E else 1) - 100
        if sh >= 0:
            q = m << sh
        elif sh > -63:
            q = (m + ((1 << -sh) >> 1)) >> -sh
        else:
            q = 0
        out.append(-q if bits >> 31 else q)
    return np.array(out, dtype=object)


def rne(x: Fraction) -> int:
    f = x.numerator // x.denominator
    d = x - f
    if d > Fraction(1, 2) or (d == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return f


def half_up(x: Fraction) -> int:
    f = (x + Fraction(1, 2))
    return f.numerator // f.denominator


def test_rint22_is_round_to_nearest_even():
    rng = np.random.default_rng(2)
    base = rng.integers(-2 ** 22, 2 ** 22, 20000)
    frac = rng.choice([0.0, 0.25, 0.5, 0.75, -0.5, 0.4999], size=base.size)
    v = (base + frac).astype(F32)
    v = np.concatenate([v, np.array([2 ** 22, -2 ** 22, 0.5, 1.5, 2.5, -0.5, -1.5, 0.0], F32)])
    v = v[np.abs(v.astype(np.float64)) <= 2 ** 22]
    assert np.array_equal(rint22(v), np.rint(v.astype(np.float64)).astype(np.int64))


def test_rint35_is_round_to_nearest_even():
    rng = np.random.default_rng(3)
    v = (rng.uniform(-1, 1, 50000) * np.ldexp(1.0, rng.integers(0, 36, 50000))).astype(F32)
    ties = (np.arange(-2000, 2000) + 0.5).astype(F32)
    edges = np.array([2 ** 35 - 2 ** 11, -(2 ** 35 - 2 ** 11), 2 ** 24 + 2, 2 ** 24 - 0.5, 4095.5, 4096.5,
                      8191.5, 8192.5, 12287.5], F32)
    v = np.concatenate([v, ties, edges])
    v = v[np.abs(v.astype(np.float64)) < 2 ** 35]
    assert np.array_equal(rint35(v), np.rint(v.astype(np.float64)).astype(np.int64))


def test_ll50_is_round_half_up_of_v_times_2_50():
    rng = np.random.default_rng(4)
    v = (rng.standard_normal(20000) * np.ldexp(1.0, rng.integers(-140, 12, 20000))).astype(F32)
    sub = np.array([1, 2, 3, 0x7FFFFF, 0x400000], dtype=np.uint32).view(F32)        # subnormals
    v = np.concatenate([v, sub, -sub, np.array([0.0, 2.0 ** -50, 1.5 * 2.0 ** -50, 2.0 ** -51, 4095.0], F32)])
    v = v[np.abs(v.astype(np.float64)) < 2 ** 12]
    got = ll50(v)
    for x, g in zip(v.tolist(), got.tolist()):
        fx = Fraction(x) * 2 ** 50
        want = half_up(fx) if fx >= 0 else -half_up(-fx)
        assert g == want, (x, g, want)


def test_level_drains_recover_the_integers():
    # acc_L = a_L 2^-(16 + 8 L) (+ its FP32 rounding for the inexact level);
    # the drain scales by 2^(16 + 8 L) and rounds: exact for |a_0|, |a_1| <= 2^22
    # (rint22), |a_2| < 2^23.6, |a_3| <= 2^23 (rint35)
    rng = np.random.default_rng(5)
    bounds = [2 ** 22, 2 ** 22, int(3 * 2 ** 22), 2 ** 23]
    for L, bnd in enumerate(bounds):
        a = np.concatenate([rng.integers(-bnd, bnd + 1, 20000), [bnd, -bnd, 0, 1, -1]])
        acc = (a.astype(np.float64) * 2.0 ** -(16 + 8 * L)).astype(F32)
        assert np.array_equal(acc.astype(np.float64) * 2.0 ** (16 + 8 * L), a.astype(np.float64))   # exact in FP32
        scaled = (acc * F32(2.0 ** (16 + 8 * L))).astype(F32)
        got = rint22(scaled) if L < 2 else rint35(scaled)
        assert np.array_equal(got, a)


def test_int64_range_sum_does_not_overflow():
    # per chunk of 256 columns, in units of 2^-49: acc_0 / 2 <= 2^22 2^32,
    # acc_1 <= 2^22 2^25, acc_2 / 2 < 3 2^22 2^16, acc_3 <= 2^23 2^9,
    # acc_4 < 2^25; 64 chunks per 16384-column range
    per_chunk = 2 ** 54 + 2 ** 47 + 3 * 2 ** 38 + 2 ** 32 + 2 ** 25
    assert 64 * per_chunk < 2 ** 63
    # and in terms of the values: |S_ij| <= 16384 |x_i| |x_j| < 2^12 (|x| < 1/2) is 2^61 units
    assert 16384 * Fraction(1, 4) * 2 ** 49 <= 2 ** 61
