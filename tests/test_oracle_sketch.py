"""Pins for the oracle's sketch operators (Sec. 2, Table 1).

Each check compares the explicit D of oracle.sketch_operator with an
independent formulation: numpy strided slicing (injection), scipy.ndimage
1-D correlation with zero boundary (nearest neighbour) and reshape-mean
(global sketch), plus Table 1's structural facts (stencil size, n_c/n).
"""
import itertools

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
import synth
from synth import GridSpec


def _rand(m, n, seed=0):
    return np.random.default_rng(seed).standard_normal((m, n))


@pytest.mark.parametrize("N,s", [((8, 8), (2, 2)), ((12, 8), (3, 4)), ((16, 16), (4, 4)),
                                 ((4, 4, 8), (2, 2, 4)), ((9,), (3,))])
def test_injection_equals_strided_slice(N, s):
    m = 5
    A = _rand(m, int(np.prod(N)))
    Y = oracle.sketch(A, GridSpec(N=N, s=s, kind="inject"))
    g = A.reshape((m,) + tuple(reversed(N)))        # (m, [Nz,] [Ny,] Nx)
    sl = tuple(slice(sd // 2, None, sd) for sd in reversed(s))
    ref = g[(slice(None),) + sl].reshape(m, -1)
    assert np.array_equal(Y, ref)


def test_injection_s1_is_identity():
    A = _rand(3, 64)
    Y = oracle.sketch(A, GridSpec(N=(8, 8), s=(1, 1), kind="inject"))
    assert np.array_equal(Y, A)
    D = oracle.sketch_operator(GridSpec(N=(8, 8), s=(1, 1), kind="inject"))
    assert (D != __import__("scipy").sparse.identity(64)).nnz == 0


@pytest.mark.parametrize("N,s", [((8, 8), (2, 2)), ((12, 12), (3, 3)), ((32, 16), (16, 4)),
                                 ((8, 4, 8), (2, 2, 4))])
def test_fullweight_equals_separable_filter(N, s):
    m = 4
    A = _rand(m, int(np.prod(N)), seed=1)
    Y = oracle.sketch(A, GridSpec(N=N, s=s, kind="fullweight"))
    g = A.reshape((m,) + tuple(reversed(N)))
    f = g
    for ax in range(1, g.ndim):
        f = ndi.correlate1d(f, [0.25, 0.5, 0.25], axis=ax, mode="constant", cval=0.0)
    sl = tuple(slice(sd // 2, None, sd) for sd in reversed(s))
    ref = f[(slice(None),) + sl].reshape(m, -1)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("N,s", [((8, 8), (2, 2)), ((12, 6), (3, 2)), ((4, 4, 4), (2, 2, 2))])
def test_blockavg_equals_reshape_mean(N, s):
    m = 3
    A = _rand(m, int(np.prod(N)), seed=2)
    Y = oracle.sketch(A, GridSpec(N=N, s=s, kind="blockavg"))
    g = A.reshape((m,) + tuple(reversed(N)))
    shp = [m]
    for Nd, sd in zip(reversed(N), reversed(s)):
        shp += [Nd // sd, sd]
    ref = g.reshape(shp).mean(axis=tuple(range(2, 2 * len(N) + 1, 2))).reshape(m, -1)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-14)


def test_table1_structure():
    """Table 1: stencil size 1 / (2d+1 per axis) / s and the fraction of the
    fine grid read (n_c/n for injection)."""
    N, s = (32, 32), (4, 4)
    Di = oracle.sketch_operator(GridSpec(N=N, s=s, kind="inject")).tocsc()
    Df = oracle.sketch_operator(GridSpec(N=N, s=s, kind="fullweight")).tocsc()
    Db = oracle.sketch_operator(GridSpec(N=N, s=s, kind="blockavg")).tocsc()
    assert set(np.diff(Di.indptr)) == {1}
    assert set(np.diff(Df.indptr)) == {9}            # 3 per axis in 2-D
    assert set(np.diff(Db.indptr)) == {16}
    assert len(np.unique(Di.indices)) / 1024 == 64 / 1024
    for D in (Di, Df, Db):
        np.testing.assert_allclose(np.asarray(D.sum(axis=0)).ravel(), 1.0)


def test_fullweight_s2_boundary_ghost_is_zero():
    """s = 2: the last cell's +1 neighbour is outside the grid and drops out."""
    D = oracle.restriction_1d(6, 2, "fullweight").toarray()
    assert D.shape == (6, 3)
    np.testing.assert_array_equal(D[:, 2], [0, 0, 0, 0, 0.25, 0.5])    # centre 5, ghost at 6
    np.testing.assert_array_equal(D[:, 0], [0.25, 0.5, 0.25, 0, 0, 0])


def test_brute_force_tiny_grid():
    """4x4 -> 2x2, m = 6: every entry of D from the per-point definition by loops."""
    m, N, s = 6, 4, 2
    A = _rand(m, N * N, seed=3)
    for kind in ("inject", "fullweight", "blockavg"):
        D = np.zeros((N * N, 4))
        for yc, xc, y, x in itertools.product(range(2), range(2), range(N), range(N)):
            def w(i, jc):
                c = s * jc + s // 2
                if kind == "inject":
                    return 1.0 if i == c else 0.0
                if kind == "fullweight":
                    return {0: 0.5, 1: 0.25, -1: 0.25}.get(i - c, 0.0)
                return 1.0 / s if s * jc <= i < s * jc + s else 0.0
            D[y * N + x, yc * 2 + xc] = w(x, xc) * w(y, yc)
        Y = oracle.sketch(A, GridSpec(N=(N, N), s=(s, s), kind=kind))
        np.testing.assert_allclose(Y, A @ D, rtol=0, atol=1e-14)


def test_subsample_index_matches_injection():
    g = GridSpec(N=(16, 8), s=(4, 2), kind="inject")
    I = oracle.subsample_index(g)
    A = _rand(3, 128, seed=4)
    np.testing.assert_array_equal(A[:, I], oracle.sketch(A, g))
    np.testing.assert_array_equal(oracle.subsample(A, g), A[:, I])


def test_batch_recipe_is_seeded_and_valid():
    """The batching workload's recipe: deterministic per seed, every factor
    divides its grid, k <= min(m, l), both field types present."""
    a = synth.batch_specs(count=256, seed=3)
    b = synth.batch_specs(count=256, seed=3)
    assert a == b
    assert len(a) == 256 and {x.field for x in a} == {"heat", "blob"}
    for x in a:
        assert x.N in (32, 64, 128, 256) and x.N % x.s == 0 and 50 <= x.m <= 2000
        assert 1 <= x.k <= min(x.m, x.l)
