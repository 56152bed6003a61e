"""Pins of the SPC-ID / SPC-ID-ERR oracle (oracle/spc.py) against facts the
paper and the mathematics fix, independent of its own code path."""
import numpy as np
import pytest

import oracle
import oracle.spc as spc
import synth
from synth import GridSpec


def _blob(m=60, N=32, s=4, seed=3):
    A = synth.blob_field(m, N, 6, seed, 1e-5, "f64")
    Ac = oracle.sketch(A, GridSpec((N, N), (s, s), "fullweight"))
    return A, Ac


def test_lifting_operator_is_the_truncated_pseudoinverse_solution():
    """The paper's simplification T_r = A_c^+ U_r U_r^T A_f, computed through
    a pseudo-inverse of the rank-r truncation instead of H."""
    A, Ac = _blob()
    r = 14
    T = spc.lifting_operator(A, Ac, r)
    U, s, Vt = np.linalg.svd(Ac, full_matrices=False)
    Acr = (U[:, :r] * s[:r]) @ Vt[:r]                  # rank-r truncation: A_c^+ U_r U_r^T = (A_c)_r^+
    T2 = np.linalg.pinv(Acr, rcond=1e-10) @ A
    # the H route applies S_c^+ twice to A_c^T A_f: rounding grows with (s_1 / s_r)^2
    kappa2 = (s[0] / s[r - 1]) ** 2
    assert kappa2 > 1e4                                # a case where the route matters
    assert np.allclose(T, T2, rtol=0, atol=100 * np.finfo(float).eps * kappa2 * np.abs(T2).max())


def test_exact_rank_k_field_is_recovered():
    """rank A_f = k with rank A_c = k: range(A_c) = range(A_f), the coarse ID
    is exact, and P_c A_c(J,:) T_k = U_k U_k^T A_f = A_f."""
    m, N, k = 40, 16, 5
    rng = np.random.default_rng(0)
    x = (np.arange(N) + 0.5) / N
    modes = [np.outer(np.sin((a + 1) * np.pi * x), np.cos(b * np.pi * x)).ravel()
             for a, b in [(0, 0), (1, 0), (0, 1), (2, 1), (1, 2)]]
    A = rng.standard_normal((m, k)) @ np.stack(modes)
    Ac = oracle.sketch(A, GridSpec((N, N), (2, 2), "fullweight"))
    assert np.linalg.matrix_rank(Ac) == k
    J, P, Sf, _ = spc.spc_id(A, Ac, k, k)
    assert np.linalg.norm(A - P @ Sf) <= 1e-11 * np.linalg.norm(A)


def test_identity_sketch_reduces_to_the_plain_row_id():
    """D = I (injection with s = 1): A_c = A_f, and with r = rank the lift
    T_r = V_r V_r^T keeps every row of A_f, so SPC-ID is the row ID of A_f."""
    A, _ = _blob(m=30, N=16)
    Ac = oracle.sketch(A, GridSpec((16, 16), (1, 1), "inject"))
    assert np.array_equal(Ac, A)
    rank = np.linalg.matrix_rank(A, tol=1e-12 * np.linalg.norm(A, 2))
    k = 8
    J, P, Sf, _ = spc.spc_id(A, Ac, k, rank)
    Jd, Pd, _ = oracle.row_id(A, k)
    assert np.array_equal(J, Jd)
    assert np.allclose(P @ Sf, Pd @ A[Jd], atol=1e-10 * np.abs(A).max())


def test_eps_closed_form_for_the_identity_sketch():
    """A_c = A_f: eps(tau) = lambda_max((1 - tau) A A^T) = (1 - tau) s_1^2 for
    tau <= 1 and (1 - tau) lambda_min(A A^T) above; lambda_min = 0 when m > n."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((12, 7))
    s = np.linalg.svd(A, compute_uv=False)
    taus = [0.0, 0.5, 1.0, 1.5, 3.0]
    e = spc.eps_exact(A, A, taus)
    want = [(1 - t) * s[0] ** 2 if t <= 1 else 0.0 for t in taus]
    assert np.allclose(e, want, atol=1e-10 * s[0] ** 2)


def test_eps_hat_special_cases():
    """c = 1 keeps every row: eps_hat = eps.  tau = 0: c * s_max(B_f)^2.
    The rows kept are 1-based multiples of c."""
    A, Ac = _blob()
    taus = [0.0, 0.01, 0.1, 1.0]
    assert np.allclose(spc.eps_hat(A, Ac, 1, taus), spc.eps_exact(A, Ac, taus), rtol=1e-12, atol=0)
    c = 4
    J = spc.subsample_rows(A.shape[0], c)
    assert J[0] == 3 and np.all(np.diff(J) == c) and len(J) == A.shape[0] // c
    e0 = spc.eps_hat(A, Ac, c, [0.0])[0]
    assert np.isclose(e0, c * np.linalg.svd(A[J], compute_uv=False)[0] ** 2, rtol=1e-12)


@pytest.mark.parametrize("k", [4, 8, 12])
def test_theorem_bound_holds(k):
    """||A_f - A_hat||_2 <= the theorem's bound with the exact eps(tau), for
    every r in [k, rank] on a tau grid (hard check)."""
    A, Ac = _blob(m=50, N=32, s=4, seed=7)
    taus = np.geomspace(1e-3, 1e2, 16)
    eps = spc.eps_exact(A, Ac, taus)
    s = np.linalg.svd(Ac, compute_uv=False)
    rank = int(np.sum(s > 1e-12 * s[0]))
    J, P, _ = oracle.row_id(Ac, k)
    e_id = np.linalg.norm(Ac - P @ Ac[J], 2)
    for r in range(k, min(rank, k + 6) + 1):
        _, _, Sf, _ = spc.spc_id(A, Ac, k, r)
        err = np.linalg.norm(A - P @ Sf, 2)
        for t, e in zip(taus, eps):
            s_next = s[r] if r < rank else 0.0
            b = np.sqrt(max(e + t * s_next ** 2, 0)) + e_id * np.sqrt(max(t + e / s[r - 1] ** 2, 0))
            assert err <= b * (1 + 1e-9), (r, t)
    bound, _, _ = spc.spc_bound(Ac, J, P, taus, eps, k)
    assert np.isfinite(bound)


def test_spc_svd_full_rank_sketch_matches_alg3_as_printed():
    """A sketch of full column rank (r = l): the U_r form of Alg. 3 and the
    literal QR(A_c), H R_c^-1 route give the same rank-k factors."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((40, 64)) @ np.diag(0.8 ** np.arange(64)) @ rng.standard_normal((64, 256))
    Ac = oracle.sketch(A, GridSpec((16, 16), (4, 4), "blockavg"))     # l = 16, full column rank
    assert np.linalg.matrix_rank(Ac) == 16
    U1, s1, V1 = spc.spc_svd(A, Ac, 6, 16)
    U2, s2, V2 = spc.spc_svd_qr(A, Ac, 6)
    assert np.allclose(s1, s2, rtol=1e-10)
    assert np.allclose(U1 @ U1.T, U2 @ U2.T, atol=1e-9) and np.allclose(V1 @ V1.T, V2 @ V2.T, atol=1e-9)


def test_spc_svd_recovers_exact_rank_k_data():
    """rank A_f = k = rank A_c: range(U_k) = range(A_f) and U S V^T = A_f."""
    m, N, k = 30, 16, 4
    rng = np.random.default_rng(9)
    x = (np.arange(N) + 0.5) / N
    modes = [np.outer(np.sin((a + 1) * np.pi * x), np.cos(b * np.pi * x)).ravel()
             for a, b in [(0, 0), (1, 0), (0, 1), (2, 1)]]
    A = rng.standard_normal((m, k)) @ np.stack(modes)
    Ac = oracle.sketch(A, GridSpec((N, N), (4, 4), "fullweight"))
    U, s, V = spc.spc_svd(A, Ac, k, k)
    assert np.linalg.norm(A - (U * s) @ V.T) <= 1e-11 * np.linalg.norm(A)
    # the singular values are A_f's own
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False)[:k], rtol=1e-10)
