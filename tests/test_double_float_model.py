"""Host model of the double-float arithmetic (pairs hi + lo of FP32 values)
that the FP64 one-sided Jacobi of the small SVD (Alg. 2) uses for its
tracked norms and rotation angle, checked in numpy FP32 without a GPU
against FP64 and exact rational references.

Every operation rounds to nearest in FP32 as the device's _rn intrinsics
do; FMA is modelled with the exact FP64 product (the error-free two-product
term is then exact; elsewhere an FP64-then-FP32 double rounding can differ
from the device's single rounding by an ulp of a correction term, far below
the bounds checked).  What must hold:

  * two-sum and the FMA two-product are error-free;
  * add (without cancellation), multiply, divide and square root are within
    2^-44 relative of the exact result;
  * the rotation angle t = sign(z) / (|z| + sqrt(1 + z^2)), z = (b - a) / 2g,
    formed from double-float a, b, g as the kernel forms it, is within
    2^-44 (1 + (a + b) / |b - a|) relative of the FP64 angle from the same
    inputs: the double-float difference b - a carries ~2^-46 (a + b), and t
    is no more sensitive than z (|dt / t| <= |dz / z|); typically ~1e-15.
    A less accurate angle only leaves a smaller off-diagonal for the next
    sweep: the kernel builds c and s so that c^2 + s^2 = 1 to FP64 rounding
    whatever the angle.
"""
from fractions import Fraction

import numpy as np

F32 = np.float32


def f(x):
    return F32(x)


def fma32(a, b, c):
    return F32(float(a) * float(b) + float(c))


def two_sum(a, b):
    s = f(a + b)
    bb = f(s - a)
    err = f(f(a - f(s - bb)) + f(b - bb))
    return s, err


def norm(s, e):
    h = f(s + e)
    return h, f(e - f(h - s))


def add(a, b):
    s, e = two_sum(a[0], b[0])
    return norm(s, f(e + f(a[1] + b[1])))


def neg(a):
    return (f(-a[0]), f(-a[1]))


def mul(a, b):
    p = f(a[0] * b[0])
    e = fma32(a[0], b[0], -p)
    return norm(p, fma32(a[0], b[1], fma32(a[1], b[0], e)))


def mul_f(a, b):
    p = f(a[0] * b)
    e = fma32(a[0], b, -p)
    return norm(p, fma32(a[1], b, e))


def div(a, b):
    q1 = f(a[0] / b[0])
    r = add(a, neg(mul_f(b, q1)))
    return norm(q1, f(r[0] / b[0]))


def sqrt(a):
    s = F32(np.sqrt(a[0]))
    p = f(s * s)
    e = fma32(s, s, -p)
    r = f(f(a[0] - p) + f(a[1] - e))
    return norm(s, f(r / f(F32(2.0) * s)))


def from_f64(x):
    hi = F32(x)
    return hi, F32(x - float(hi))


def val(a):
    return Fraction(float(a[0])) + Fraction(float(a[1]))


def rel(got, exact):
    return abs(got - exact) / abs(exact)


def test_two_sum_and_two_product_are_error_free():
    rng = np.random.default_rng(1)
    for _ in range(5000):
        a, b = F32(rng.standard_normal() * 2.0 ** rng.integers(-20, 20)), F32(rng.standard_normal())
        s, e = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))
        p = f(a * b)
        e2 = fma32(a, b, -p)
        assert Fraction(float(p)) + Fraction(float(e2)) == Fraction(float(a)) * Fraction(float(b))


def test_operations_within_2_44():
    rng = np.random.default_rng(2)
    worst = {"add": 0.0, "mul": 0.0, "div": 0.0, "sqrt": 0.0}
    for _ in range(4000):
        x = rng.uniform(0.5, 2.0) * 2.0 ** rng.integers(-30, 30)
        y = rng.uniform(0.5, 2.0) * 2.0 ** rng.integers(-30, 30)
        a, b = from_f64(x), from_f64(y)
        va, vb = val(a), val(b)
        worst["add"] = max(worst["add"], float(rel(val(add(a, b)), va + vb)))
        worst["mul"] = max(worst["mul"], float(rel(val(mul(a, b)), va * vb)))
        worst["div"] = max(worst["div"], float(rel(val(div(a, b)), va / vb)))
        s = val(sqrt(a))
        worst["sqrt"] = max(worst["sqrt"], float(abs(s * s - va) / va) / 2)      # d sqrt / sqrt = d a / 2a
    for k, w in worst.items():
        assert w <= 2.0 ** -44, (k, w)


def test_rotation_angle_within_its_cancellation_bound():
    rng = np.random.default_rng(3)
    ratios = []
    for _ in range(3000):
        # squared norms a, b and the inner product g with |g| <= sqrt(a b)
        a = rng.uniform(0.1, 10.0) * 10.0 ** rng.integers(-6, 6)
        b = rng.uniform(0.1, 10.0) * 10.0 ** rng.integers(-6, 6)
        g = rng.uniform(-1, 1) * np.sqrt(a * b) * 10.0 ** -rng.integers(0, 8)
        if g == 0.0:
            continue
        A, B, G = from_f64(a), from_f64(b), from_f64(g)
        dd = add(B, neg(A))
        zeta = div(dd, (f(F32(2.0) * G[0]), f(F32(2.0) * G[1])))
        if abs(zeta[0]) > 1e18:
            t = div((F32(0.5), F32(0.0)), zeta)
        else:
            w = sqrt(add((F32(1.0), F32(0.0)), mul(zeta, zeta)))
            den = add(neg(zeta) if zeta[0] < 0 else zeta, w)
            t = div((F32(-1.0) if zeta[0] < 0 else F32(1.0), F32(0.0)), den)
        # the FP64 angle from the same (rounded) inputs
        a64, b64, g64 = float(val(A)), float(val(B)), float(val(G))
        z = (b64 - a64) / (2 * g64)
        t64 = np.sign(z) / (abs(z) + np.sqrt(1 + z * z)) if z != 0 else 1.0
        err = abs(float(val(t)) - t64) / abs(t64)
        bound = 2.0 ** -44 * (1.0 + (a64 + b64) / abs(b64 - a64)) if b64 != a64 else 2.0 ** -44
        ratios.append(err / bound)
        assert err <= bound, (a, b, g, err, bound)
    assert np.median(ratios) < 0.1
