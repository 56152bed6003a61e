"""SPC-SVD, SPC-ID and the single-pass error estimate (oracle; test infrastructure).

Paper, Sec. 3.2, Alg. 3 (SPC-SVD).  The same single read forms A_c = A_f D and
H = A_f^T A_c; then QR(A_c) = Q_c R_c, H R_c^-1 = A_f^T Q_c, and the SVD of
(H R_c^-1)^T = Q_c^T A_f = U~ S V^T gives U = Q_c U~, S, V (rank k: the
leading k).  Reading: R_c^-1 exists only on the numerical range of A_c (the
sketch of FP32 or smooth data is numerically rank deficient), so Q_c is taken
as the leading r left singular vectors U_r of A_c, where R_c^-1 becomes
V_r S_r^-1 (A_c V_r S_r^-1 = U_r):  B = S_r^-1 V_r^T H^T = U_r^T A_f.  With r =
rank A_c = l (full column rank) this is Alg. 3 as printed (range(U_r) =
range(Q_c)); the pins check that case against the literal QR route.

Paper, Sec. 4, Alg. 5 (SPC-ID).  One read of A_f, row by row, forms

    A_c = A_f D          (m x l, the sketch)
    H   = A_f^T A_c      (n x l)

then, with the SVD A_c = U_c S_c V_c^T and U_r = U_c(:, 1:r), k <= r <= rank A_c,
the lifting operator is

    T_r = V_c S_c^+ U_c^T U_r U_r^T U_c S_c^+ V_c^T H^T        (l x n)

and, with the rank-k row ID A_c ~ P_c A_c(I_c, :),

    A_f ~ P_c A_c(I_c, :) T_r.

The paper shows T_r = A_c^+ U_r U_r^T A_f (H^T = V_c S_c U_c^T A_f); the pins
use that identity, computed another way, as a check.

Alg. 6 (SPC-ID-ERR).  Every c-th snapshot is kept while A_f is read,
B_f = A_f(J, :), B_c = A_c(J, :), and

    eps_hat(tau) = c * lambda_max(B_f B_f^T - tau B_c B_c^T)

estimates eps(tau) = lambda_max(A_f A_f^T - tau A_c A_c^T) of the error bound
(Theorem on SPC-ID):

    ||A_f - A_hat||_2 <= min over tau, k <= r <= rank A_c of
        (eps(tau) + tau s_{c,r+1}^2)^{1/2}
        + ||A_c - P_c A_c(I_c,:)||_2 (tau + eps(tau) s_{c,r}^{-2})^{1/2}.

Readings:
  * U_c, S_c, V_c: the thin SVD of A_c (min(m, l) columns).  S_c^+ inverts the
    singular values above rtol * s_1 (rtol = 1e-12) and zeroes the rest; r is
    capped at that numerical rank.
  * U_c^T U_r = [I_r; 0] by the orthonormality of U_c's columns, so the factor
    in front of H^T is V_r S_r^-2 V_r^T.  Evaluated literally, the rounding
    left in U_c^T U_r U_r^T U_c beyond the first r directions is multiplied by
    (S_c^+)^2, up to 1e24 for the directions near the cutoff; the identity is
    exact, and the oracle uses it.
  * "ID(A_c)": the row ID of A_c by CPQR of A_c^T, as in Alg. 4 (interp.row_id).
  * J of Alg. 6: the 1-based rows i with mod(i, c) = 0, i.e. the 0-based rows
    c-1, 2c-1, ...; m_c = floor(m / c), c a positive integer.
  * Alg. 6 prints "min over tau" around eps_hat, but eps(tau) falls without
    bound as tau grows whenever B_c B_c^T is definite, and the theorem's bound
    minimises over tau only together with its other terms.  eps_hat is
    therefore returned for each tau of a caller-given grid, and the bound is
    minimised over that grid and over r.
  * s_{c,r+1} = 0 for r = rank A_c.  A negative value under either square root
    (impossible in exact arithmetic, where both bound non-negative norms) is
    taken as 0.
"""
from __future__ import annotations

import numpy as np

from .interp import row_id
from .sketch import as_f64

SVD_RTOL = 1e-12


def _thin_svd(Ac: np.ndarray):
    U, s, Vt = np.linalg.svd(Ac, full_matrices=False)
    rank = int(np.sum(s > SVD_RTOL * s[0])) if s.size and s[0] > 0 else 0
    return U, s, Vt.T, rank


def lifting_operator(Af, Ac: np.ndarray, r: int, col_block: int = 1 << 15):
    """T_r (l x n): Alg. 5's formula (with U_c^T U_r = [I_r; 0]) applied to
    H^T, H accumulated from A_f in column slabs."""
    Af = as_f64(Af)
    m, n = Af.shape
    U, s, V, rank = _thin_svd(Ac)
    if not 1 <= r <= rank:
        raise ValueError(f"r = {r} outside [1, rank A_c = {rank}]")
    # the l x l factor in front of H^T: V_c S_c^+ (U_c^T U_r)(U_r^T U_c) S_c^+ V_c^T
    # with U_c^T U_r = [I_r; 0], i.e. V_r S_r^-2 V_r^T
    Vr = V[:, :r]
    mid = (Vr / s[:r] ** 2) @ Vr.T
    T = np.empty((Ac.shape[1], n))
    for c0 in range(0, n, col_block):
        Hb = Af[:, c0:c0 + col_block].T @ Ac          # rows c0.. of H = A_f^T A_c
        T[:, c0:c0 + col_block] = mid @ Hb.T
    return T


def spc_id(Af, Ac: np.ndarray, k: int, r: int):
    """Alg. 5.  Returns (J, P, S_f, T_r) with S_f = A_c(J, :) T_r, so that
    A_f ~ P S_f."""
    if r < k:
        raise ValueError("the lifting rank r must be >= k")
    T = lifting_operator(Af, Ac, r)
    J, P, _ = row_id(Ac, k)
    return J, P, Ac[J] @ T, T


def spc_svd(Af, Ac: np.ndarray, k: int, r: int, col_block: int = 1 << 15):
    """Alg. 3 with Q_c = U_r: returns (U_k, S_k, V_k) of B = S_r^-1 V_r^T H^T."""
    Af = as_f64(Af)
    n = Af.shape[1]
    U, s, V, rank = _thin_svd(Ac)
    if not 1 <= r <= rank:
        raise ValueError(f"r = {r} outside [1, rank A_c = {rank}]")
    left = V[:, :r] / s[:r]                         # R_c^-1 restricted: V_r S_r^-1 (l x r)
    B = np.empty((r, n))
    for c0 in range(0, n, col_block):
        Hb = Af[:, c0:c0 + col_block].T @ Ac        # rows c0.. of H = A_f^T A_c
        B[:, c0:c0 + col_block] = (Hb @ left).T     # (H R_c^-1)^T
    Ub, sb, Vbt = np.linalg.svd(B, full_matrices=False)
    kk = min(k, r)
    return U[:, :r] @ Ub[:, :kk], sb[:kk], Vbt[:kk].T


def spc_svd_qr(Af, Ac: np.ndarray, k: int):
    """Alg. 3 as printed, for a sketch of full column rank: QR(A_c), H R_c^-1,
    SVD of its transpose."""
    Af = as_f64(Af)
    Qc, Rc = np.linalg.qr(Ac)
    H = Af.T @ Ac
    HR = np.linalg.solve(Rc.T, H.T).T               # H R_c^-1
    Ub, sb, Vbt = np.linalg.svd(HR.T, full_matrices=False)
    return Qc @ Ub[:, :k], sb[:k], Vbt[:k].T


def subsample_rows(m: int, c: int) -> np.ndarray:
    """J of Alg. 6 (0-based)."""
    if c < 1:
        raise ValueError("c >= 1")
    return np.arange(c - 1, (m // c) * c, c)


def eps_exact(Af, Ac: np.ndarray, taus) -> np.ndarray:
    """eps(tau) = lambda_max(A_f A_f^T - tau A_c A_c^T)."""
    Af = as_f64(Af)
    Gf, Gc = Af @ Af.T, Ac @ Ac.T
    return np.array([np.linalg.eigvalsh(Gf - t * Gc)[-1] for t in taus])


def eps_hat(Af, Ac: np.ndarray, c: int, taus) -> np.ndarray:
    """Alg. 6: c * lambda_max(B_f B_f^T - tau B_c B_c^T) for each tau."""
    J = subsample_rows(Ac.shape[0], c)
    Bf, Bc = as_f64(Af)[J], Ac[J]
    Gf, Gc = Bf @ Bf.T, Bc @ Bc.T
    return np.array([c * np.linalg.eigvalsh(Gf - t * Gc)[-1] for t in taus])


def spc_bound(Ac: np.ndarray, J: np.ndarray, P: np.ndarray, taus, eps, k: int):
    """The theorem's right-hand side, minimised over the tau grid (with its
    eps values) and over k <= r <= rank A_c.  Returns (bound, tau, r)."""
    s = np.linalg.svd(Ac, compute_uv=False)
    rank = int(np.sum(s > SVD_RTOL * s[0]))
    e_id = np.linalg.norm(Ac - P @ Ac[J], 2)
    best = (np.inf, None, None)
    for t, e in zip(taus, eps):
        for r in range(k, rank + 1):
            s_next = s[r] if r < rank else 0.0
            b = np.sqrt(max(e + t * s_next ** 2, 0.0)) + e_id * np.sqrt(max(t + e / s[r - 1] ** 2, 0.0))
            if b < best[0]:
                best = (b, t, r)
    return best
