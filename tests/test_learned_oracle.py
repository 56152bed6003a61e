"""CPU pins of the learned proposal's oracle (oracle/learned.py) and of the
stored training set (tests/golden/learned_set.npz, written by
tests/golden/make_learned_set.py from synth + oracle only)."""
import os

import numpy as np
import pytest

import oracle.learned as L

HERE = os.path.dirname(os.path.abspath(__file__))
SET = os.path.join(HERE, "golden", "learned_set.npz")


def _params(seed):
    rng = np.random.default_rng(seed)
    return {"W1": rng.standard_normal((L.N_HID, L.N_IN)) * 0.2, "b1": rng.standard_normal(L.N_HID) * 0.1,
            "W2": rng.standard_normal((L.N_HID, L.N_HID)) * 0.1, "b2": rng.standard_normal(L.N_HID) * 0.1,
            "W3": rng.standard_normal((L.N_OUT, L.N_HID)) * 0.1, "b3": rng.standard_normal(L.N_OUT) * 0.1}


def test_mlp_gradient_matches_central_differences():
    """The analytic gradient against central differences of the loss (unrounded
    weights, so the loss is smooth), on a few entries of every tensor."""
    p = _params(0)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((9, L.N_IN))
    y = rng.integers(0, L.N_OUT, 9)
    _, g = L.mlp_loss_grad(p, X, y, round_weights=False)
    h = 1e-6
    for name in p:
        flat = p[name].ravel()
        for idx in rng.choice(flat.size, 5, replace=False):
            q = {k: v.copy() for k, v in p.items()}
            q[name].ravel()[idx] += h
            lp, _ = L.mlp_loss_grad(q, X, y, round_weights=False)
            q[name].ravel()[idx] -= 2 * h
            lm, _ = L.mlp_loss_grad(q, X, y, round_weights=False)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].ravel()[idx]) <= 1e-6 + 1e-5 * abs(fd), (name, idx)


def test_mlp_uses_bf16_weights_and_pack_roundtrips():
    p = _params(2)
    X = np.random.default_rng(3).standard_normal((4, L.N_IN))
    z_r, _ = L.mlp_forward(p, X)
    q = {k: (L.bf16_round(v) if k.startswith("W") else v) for k, v in p.items()}
    z_q, _ = L.mlp_forward(q, X, round_weights=False)
    assert np.array_equal(z_r, z_q)
    flat = L.pack(p)
    assert all(np.array_equal(L.unpack(flat)[k], p[k]) for k in p)


def test_range_basis_and_label_on_an_exact_rank_field():
    """A rank-3 field captured by every configuration: label 0, tiny errors."""
    N, m = 32, 40
    rng = np.random.default_rng(4)
    x = (np.arange(N) + 0.5) / N
    modes = [np.outer(np.sin((a + 1) * np.pi * x), np.sin((b + 1) * np.pi * x)).ravel() for a, b in
             [(0, 0), (1, 0), (0, 1)]]
    A = rng.standard_normal((m, 3)) @ np.stack(modes)
    y, errs = L.label(A, N)
    assert y == 0 and max(errs) < 1e-10
    # features: three singular values, the rest missing; rank 3 of min(m, l) = min(40, 16)
    f = L.features(A, N)
    assert np.all(f[:3] > -1.0) and f[0] == 0.0 and np.all(f[3:L.N_SIGMA] == -1.0)
    assert np.all(np.diff(f[:3]) <= 0.0)              # a pivoted R's diagonal does not increase
    assert f[L.N_SIGMA + 2] == 3 / 16 and f[L.N_SIGMA] == 5 / 8


@pytest.mark.skipif(not os.path.exists(SET), reason="learned_set.npz not generated")
def test_stored_set_is_consistent():
    d = np.load(SET)
    for split in ("train", "test"):
        X, y, E = d[f"X_{split}"], d[f"y_{split}"], d[f"err_{split}"]
        assert X.shape[1] == L.N_IN and E.shape[1] == L.N_OUT and len(X) == len(y) == len(E)
        assert np.all((X >= -1.0) & (X <= 1.5))
        for yi, e in zip(y, E):
            ok = np.nonzero(e <= 1e-3)[0]
            assert yi == (ok[0] if ok.size else L.N_OUT - 1)
    assert len(set(map(tuple, d["meta_train"][:, -1:])) & set(map(tuple, d["meta_test"][:, -1:]))) == 0


def test_first_adam_step_moves_each_parameter_by_lr():
    """With zero moments, the bias-corrected first step is lr * g / (|g| + eps):
    a move of lr against the sign of every gradient entry much larger than eps."""
    rng = np.random.default_rng(5)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50) + np.sign(rng.standard_normal(50)) * 0.1
    q, m1, m2 = L.adam_step(p, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(p - q, 1e-3 * np.sign(g), rtol=1e-6, atol=0)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)
    # a constant gradient keeps the step at lr (the bias corrections cancel the averages' start)
    for t in range(2, 6):
        q2, m1, m2 = L.adam_step(q, g, m1, m2, t, 1e-3)
        assert np.allclose(q - q2, 1e-3 * np.sign(g), rtol=1e-6, atol=0)
        q = q2
