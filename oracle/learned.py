"""FP64 oracle of the learned sketch proposal (test infrastructure).

The proposal (an addition to the paper's method) chooses, per
matrix, the cheapest sketch configuration of the method that captures A_f to
a relative Frobenius tolerance:

  configurations, cheapest first (full weighting per axis factor s, C-PWR q
  passes on the 2x injection subsample):
      (s, q) = (8, 0), (8, 1), (4, 0), (4, 1), (2, 0), (2, 1)
  a configuration passes when the range finder's basis Q (QR(Y) for q = 0,
  the re-orthonormalised C-PWR iterate for q = 1, rtol 1e-6) captures A:
      ||A - Q Q^T A||_F / ||A||_F <= tol        (tol = 1e-3)
  label = index of the cheapest passing configuration (the last one if none).

Features come from the cheapest configuration's range finder, which the
adaptive enlargement runs first anyway: Y = A D (full weighting, s = 8), its
pivoted QR Y P = Q R stopped at rtol 1e-6 after r steps, and the leading 64
diagonal entries d_i = |R_ii| (non-increasing; the rank-revealing part of
the factorization) as log10(d_i / d_0) clipped to [-6, 0] and divided by 6
(missing values -1); then log2(N) / 8, log2(m) / 11 and r / min(m, l): 67
numbers.

The MLP (3 layers, width 128, ReLU, softmax cross-entropy over the 6
configurations) is restated in float64 with its weights rounded to BF16 as
the GPU stores them: forward, loss and the exact gradient; Adam restated
from its definition.
"""
from __future__ import annotations

import numpy as np

from .sketch import as_f64, sketch, subsample
from .cpqr import cpqr
from .rangefinder import range_find
from .cpwr import cpwr

CONFIGS = [(8, 0), (8, 1), (4, 0), (4, 1), (2, 0), (2, 1)]
FEATURE_RTOL = 1e-6            # the range finder's tolerance in every configuration
N_SIGMA = 64
N_IN, N_HID, N_OUT = N_SIGMA + 3, 128, len(CONFIGS)


def grids_for(N: int, s: int, q: int):
    """(sketch grid, C-PWR subsample grid or None) of configuration (s, q) on an N x N grid."""
    from synth import GridSpec
    g = GridSpec((N, N), (s, s), "fullweight")
    gram = GridSpec((N, N), (2, 2), "inject") if q > 0 else None
    return g, gram


def range_basis(A, N: int, s: int, q: int, rtol: float = 1e-6):
    """The method's orthonormal basis for configuration (s, q)."""
    g, gram = grids_for(N, s, q)
    Y = sketch(A, g)
    if q == 0:
        Q, _ = range_find(Y, rtol)
        return Q
    G, _ = cpwr(Y, subsample(A, gram), q, True, rtol)
    return G


def projection_error(A, Q) -> float:
    """||A - Q Q^T A||_F / ||A||_F."""
    A = as_f64(A)
    R = A - Q @ (Q.T @ A)
    return float(np.linalg.norm(R) / np.linalg.norm(A))


def features(A, N: int) -> np.ndarray:
    A = as_f64(A)
    g, _ = grids_for(N, CONFIGS[0][0], 0)
    Y = sketch(A, g)
    _, R, _, r, _ = cpqr(Y, rtol=FEATURE_RTOL)
    f = -np.ones(N_IN)
    d = np.abs(np.diag(R)[: min(r, N_SIGMA)])
    if d.size and d[0] > 0:
        v = np.log10(np.maximum(d / d[0], 1e-300))
        f[: d.size] = np.clip(v, -6.0, 0.0) / 6.0
    m, l = A.shape[0], Y.shape[1]
    f[N_SIGMA] = np.log2(N) / 8.0
    f[N_SIGMA + 1] = np.log2(m) / 11.0
    f[N_SIGMA + 2] = r / min(m, l)
    return f


def label(A, N: int, tol: float = 1e-3):
    """(label, per-configuration projection errors)."""
    errs = [projection_error(A, range_basis(A, N, s, q, FEATURE_RTOL)) for (s, q) in CONFIGS]
    passing = [i for i, e in enumerate(errs) if e <= tol]
    return (passing[0] if passing else len(CONFIGS) - 1), errs


SHAPES = (("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,)))


def unpack(p: np.ndarray) -> dict:
    """The flat parameter layout (W1 | b1 | W2 | b2 | W3 | b3, row-major) as named arrays."""
    out, off = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.ravel(d[k]) for k, _ in SHAPES])


# ---------------------------------------------------------------------------
# the MLP in float64
def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (RNE) and back to float64."""
    from synth import to_bf16_bits, bf16_bits_to_f64
    return bf16_bits_to_f64(to_bf16_bits(np.asarray(x, dtype=np.float64)))


def mlp_forward(params: dict, X: np.ndarray, round_weights: bool = True):
    """logits and the activations; weights used as their BF16 roundings
    (round_weights=False uses them as given: the finite-difference pin)."""
    rnd = bf16_round if round_weights else (lambda w: np.asarray(w, dtype=np.float64))
    W1, W2, W3 = (rnd(params[k]) for k in ("W1", "W2", "W3"))
    z1 = X @ W1.T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + params["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3.T + params["b3"]
    return z3, (X, z1, h1, z2, h2)


def mlp_loss_grad(params: dict, X: np.ndarray, y: np.ndarray, round_weights: bool = True):
    """Mean softmax cross-entropy and its exact gradient (w.r.t. the BF16 weights and the biases)."""
    rnd = bf16_round if round_weights else (lambda w: np.asarray(w, dtype=np.float64))
    W2, W3 = rnd(params["W2"]), rnd(params["W3"])
    z3, (X, z1, h1, z2, h2) = mlp_forward(params, X, round_weights)
    B = X.shape[0]
    zmax = z3.max(axis=1, keepdims=True)
    e = np.exp(z3 - zmax)
    p = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(p[np.arange(B), y])))
    d3 = p.copy()
    d3[np.arange(B), y] -= 1.0
    d3 /= B
    g = {"W3": d3.T @ h2, "b3": d3.sum(axis=0)}
    d2 = (d3 @ W3) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return loss, g


def adam_step(p: np.ndarray, g: np.ndarray, m1: np.ndarray, m2: np.ndarray, step: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba, 2015) on the flat parameters: moment
    averages, bias corrections 1 - beta^step, p -= lr m1_hat / (sqrt(m2_hat) + eps).
    Returns the new (p, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    mh = m1 / (1.0 - beta1 ** step)
    vh = m2 / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
