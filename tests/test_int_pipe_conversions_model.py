"""Host model of the integer-pipe conversions the FP64 kernels use instead of
the FP64 pipe's conversion instructions (the sketch's FP32 loads, the
double-float Jacobi, the pivoted factorisations' reciprocal square roots),
checked in numpy without a GPU against numpy's own conversions.

  * widen_f32: exponent rebiased by 896 and the 23 fraction bits shifted up
    by 29 is the exact FP64 value of every normal FP32 number and of +-0;
  * split_f64_f2, for 2^-74 <= |x| < 2^127: hi (x's sign, exponent and top 23
    fraction bits) is x truncated toward zero to FP32, lo (the low 29 fraction
    bits as an integer, converted with round-to-nearest and scaled by
    2^(e - 52) through its exponent field) is the round-to-nearest FP32 of
    x - hi, and hi + lo is within 2^-47 |x| of x;
  * the pivot keys: non-negative doubles order as their bit patterns.
"""
import numpy as np

F32 = np.float32


def widen_f32_bits(f):
    u = np.asarray(f, dtype=F32).view(np.uint32).astype(np.uint64)
    e = (u >> np.uint64(23)) & np.uint64(0xFF)
    sign = (u & np.uint64(0x80000000)) << np.uint64(32)
    normal = sign | ((e + np.uint64(896)) << np.uint64(52)) | ((u & np.uint64(0x7FFFFF)) << np.uint64(29))
    zero = sign
    out = np.where((e >= 1) & (e <= 254), normal, zero)
    return out.view(np.float64)


def split_f64_f2_model(x):
    u = np.asarray(x, dtype=np.float64).view(np.uint64)
    e = ((u >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023
    assert np.all((e >= -74) & (e < 127))
    sign = ((u >> np.uint64(32)) & np.uint64(0x80000000)).astype(np.uint32)
    m = u & np.uint64(0xFFFFFFFFFFFFF)
    hi = (sign | ((e + 127).astype(np.uint32) << 23) | (m >> np.uint64(29)).astype(np.uint32)).view(F32)
    rest = (m & np.uint64(0x1FFFFFFF)).astype(np.uint64)
    rf = rest.astype(np.float64).astype(F32)                    # integer -> FP32, round to nearest
    lo_bits = sign | (rf.view(np.uint32) - ((52 - e).astype(np.uint32) << 23))
    lo = np.where(rest != 0, lo_bits.view(F32), F32(0.0))
    return hi, lo


def test_widen_f32_is_exact_for_normals_and_zeros():
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(F32)
    e = (bits >> 23) & 0xFF
    keep = ((e >= 1) & (e <= 254)) | ((bits & 0x7FFFFFFF) == 0)
    f = np.concatenate([f[keep], np.array([0.0, -0.0, 1.0, -1.0, np.finfo(F32).max, np.finfo(F32).tiny], F32)])
    got = widen_f32_bits(f)
    ref = f.astype(np.float64)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))      # bit for bit, signed zeros too


def test_split_f64_f2_truncates_then_rounds():
    rng = np.random.default_rng(8)
    x = rng.standard_normal(200000) * np.ldexp(1.0, rng.integers(-74, 127, 200000))
    x = np.concatenate([x, np.ldexp(1.0, np.arange(-74, 127)), -np.ldexp(1.0 + 2.0 ** -52, np.arange(-74, 126))])
    e = np.frexp(np.abs(x))[1] - 1
    x = x[(e >= -74) & (e < 127)]
    hi, lo = split_f64_f2_model(x)
    hd = hi.astype(np.float64)
    # hi is x truncated toward zero to FP32: |hi| <= |x| with the same sign,
    # and |x - hi| below one FP32 ulp of hi
    assert np.all(np.abs(hd) <= np.abs(x)) and np.all(np.sign(hd) == np.sign(x))
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    assert np.all(np.abs(x - hd) < ulp)
    # lo is the round-to-nearest FP32 of the exact remainder
    rem = x - hd                                                          # exact in FP64
    assert np.array_equal(lo, rem.astype(F32))
    assert np.all(np.abs(x - (hd + lo.astype(np.float64))) <= 2.0 ** -47 * np.abs(x))


def test_nonnegative_doubles_order_as_their_bits():
    rng = np.random.default_rng(9)
    a = np.abs(rng.standard_normal(5000) * np.ldexp(1.0, rng.integers(-1070, 1020, 5000)))
    a = np.concatenate([a, [0.0, 5e-324, np.finfo(np.float64).max, np.inf]])
    k = a.view(np.int64)
    order_v = np.argsort(a, kind="stable")
    order_k = np.argsort(k, kind="stable")
    assert np.array_equal(a[order_v], a[order_k])
