"""Host model of the exact-slice Gram (the tensor-core Gram of B in the small
SVD, Alg. 2): the slicing, the level accounting and the exactness ranges its
kernel relies on, checked in numpy without a GPU.

What must hold:
  * x = b 2^-(e+1) with max|b| < 2^e has |x| < 1/2, and the six slices cut by
    the FP32 magic-number rounding are integers times 2^-8(t+1) with
    |integer| <= 128, so their FP32 bits have zero low halves (exact BF16);
    x - sum(slices) is within 2^-49;
  * over a chunk of 256 columns every exactly-summed level stays below 2^24
    of its units, at the largest slice values too (acc_0, acc_1 <= 2^22,
    acc_2 = X_02 + X_20 + X_11 <= 3 * 2^22, acc_3 = X_03 + X_12 <= 2^23);
  * S = acc_0/2 + acc_1 + acc_2/2 + acc_3 + acc_4 gives S + S^T equal to the
    sum of every slice product of level <= 5, in exact integer arithmetic;
  * the Gram from the kept levels is within 2^-46 of sum_k |b_ik b_jk| of the
    correctly rounded Gram off the diagonal; on it the dropped terms are
    squares and the kept levels fall short by a one-signed ~2^-45 (the reason
    the diagonal is summed apart, from x^2).
"""
import math

import numpy as np

F32 = np.float32
MAGIC = [F32(1.5 * 2.0 ** (15 - 8 * t)) for t in range(6)]
LEVEL_UNIT = [2.0 ** (-8 * (L + 2)) for L in range(11)]


def row_scale(b):
    m = float(np.max(np.abs(b))) if b.size else 0.0
    e = math.frexp(m)[1] if m > 0 else 0          # m < 2^e
    return e


def slice_row(b):
    """x = b 2^-(e+1) and its six slices (FP32 arithmetic, as the kernel)."""
    e = row_scale(b)
    x = (b.astype(np.float64) * 2.0 ** -(e + 1)).astype(F32)
    assert np.array_equal(x.astype(np.float64), b.astype(np.float64) * 2.0 ** -(e + 1))   # exact scaling
    rem = x.copy()
    sl = []
    for t in range(6):
        s = (rem + MAGIC[t]) - MAGIC[t]           # numpy float32: round to nearest even each step
        rem = rem - s
        sl.append(s)
    return e, x, sl


def ints(s, t):
    return np.rint(s.astype(np.float64) * 2.0 ** (8 * (t + 1))).astype(np.int64)


def test_slices_are_exact_bf16_integers():
    rng = np.random.default_rng(3)
    rows = [rng.standard_normal(4096).astype(F32),
            (rng.standard_normal(4096) * np.ldexp(1.0, rng.integers(-30, 31, 4096))).astype(F32),
            np.full(256, F32(2 ** 20 - 1)), np.full(256, F32(-0.9999999)), np.zeros(64, F32)]
    for b in rows:
        e, x, sl = slice_row(b)
        assert np.all(np.abs(x) < 0.5)
        for t, s in enumerate(sl):
            k = ints(s, t)
            assert np.array_equal(k.astype(np.float64) * 2.0 ** (-8 * (t + 1)), s.astype(np.float64))
            assert np.max(np.abs(k)) <= 128
            assert np.all((s.view(np.uint32) & 0xFFFF) == 0)           # the BF16 bits are the FP32 bits
        resid = x.astype(np.float64) - sum(s.astype(np.float64) for s in sl)
        assert np.max(np.abs(resid)) <= 2.0 ** -49


def chunk_levels(K):
    """Integer level sums over one chunk for slice-integer matrices K[t] (r x c)."""
    X = {(s, t): K[s] @ K[t].T for s in range(6) for t in range(6)}
    acc0 = X[0, 0]
    acc1 = X[0, 1]
    acc2 = X[0, 2] + X[2, 0] + X[1, 1]
    acc3 = X[0, 3] + X[1, 2]
    return X, acc0, acc1, acc2, acc3


def test_exact_accumulators_stay_below_2_24_per_chunk():
    c = 256
    # the worst case: every slice at +-128 with one sign, and random slices
    for K in ([np.full((4, c), 128, np.int64) for _ in range(6)],
              [np.random.default_rng(t).integers(-128, 129, (4, c)) for t in range(6)]):
        _, a0, a1, a2, a3 = chunk_levels(K)
        assert np.max(np.abs(a0)) <= 2 ** 22
        assert np.max(np.abs(a1)) <= 2 ** 22
        assert np.max(np.abs(a2)) < 2 ** 24 and np.max(np.abs(a2)) <= 3 * 2 ** 22
        assert np.max(np.abs(a3)) <= 2 ** 23


def test_symmetric_level_identity():
    rng = np.random.default_rng(5)
    K = [rng.integers(-128, 129, (7, 300)) for _ in range(6)]
    X, a0, a1, a2, a3 = chunk_levels(K)
    # in units of 2^-8 (L+2) of each level; acc_4 = X_04 + X_13 + X_22/2 + X_05 + X_14 + X_23
    # scaled to level-5 units (times 2 for the half) to stay in integers
    two_S = {0: a0, 1: 2 * a1, 2: a2, 3: 2 * a3}
    two_acc4_l5 = 2 * (X[0, 4] + X[1, 3]) * 256 + X[2, 2] * 256 + 2 * (X[0, 5] + X[1, 4] + X[2, 3])
    # S + S^T per level equals the full sum of the ordered pairs of that level
    for L in range(4):
        full = sum(X[s, L - s] for s in range(L + 1))
        assert np.array_equal(two_S[L] + two_S[L].T, 2 * full)
    full45 = sum(X[s, 4 - s] for s in range(5)) * 256 + sum(X[s, 5 - s] for s in range(6))
    assert np.array_equal(two_acc4_l5 + two_acc4_l5.T, 2 * full45)


def test_model_gram_accuracy():
    rng = np.random.default_rng(11)
    r, n = 6, 3000
    B = (rng.standard_normal((r, n)) * np.logspace(0, -3, r)[:, None]).astype(F32)
    es, Ks = [], []
    for i in range(r):
        e, _, sl = slice_row(B[i])
        es.append(e)
        Ks.append([ints(s, t) for t, s in enumerate(sl)])
    K = [np.stack([Ks[i][t] for i in range(r)]) for t in range(6)]
    # every kept level (s + t <= 5) exactly, in integers of the level's unit
    G = np.zeros((r, r))
    for L in range(6):
        lev = sum(K[s] @ K[L - s].T for s in range(L + 1))
        G += lev.astype(np.float64) * LEVEL_UNIT[L]
    scale = np.ldexp(1.0, np.array(es) + 1)
    G *= np.outer(scale, scale)
    b = B.astype(np.float64)
    ref = np.array([[math.fsum(b[i] * b[j]) for j in range(r)] for i in range(r)])
    bound = np.abs(b) @ np.abs(b).T
    off = ~np.eye(r, dtype=bool)
    assert np.max((np.abs(G - ref) / bound)[off]) <= 2.0 ** -46
    # on the diagonal the dropped terms (X_33, level 6, ...) are squares: the
    # kept levels fall short by a one-signed ~2^-45, which is why the kernel
    # sums G_ii = sum_k x_ik^2 apart
    short = np.diag(ref - G) / np.diag(ref)
    assert np.all(short > 0) and np.all(short < 2.0 ** -43)
    diag = np.array([math.fsum((b[i] * 2.0 ** -(es[i] + 1)) ** 2) for i in range(r)]) * scale ** 2
    assert np.max(np.abs(diag - np.diag(ref)) / np.diag(ref)) <= 2.0 ** -50
