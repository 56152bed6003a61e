"""Learned sketch proposal on the GPU, against the FP64 oracle (oracle/learned.py).

1. The MLP kernels: BF16 weight rounding (bit-exact), logits, loss and the
   gradient of every parameter, and the Adam update.
2. The features of the first configuration's basis, GPU against oracle, on
   matrices of the stored set's recipe.
3. Training on the stored set by the GPU kernels, then the learned start
   against the plain adaptive enlargement on held-out matrices: the accepted
   bases meet the tolerance, the learned start tries fewer configurations and
   takes less time.
"""
import os
import sys

import numpy as np
import pytest

import oracle.learned as L
import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SET = os.path.join(HERE, "golden", "learned_set.npz")
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_learned_set as recipe  # noqa: E402  (synth-only matrix recipe of the stored set)

TOL = 1e-3


def _torch():
    import torch
    return torch


def _random_params(seed):
    rng = np.random.default_rng(seed)
    d = {"W1": rng.standard_normal((L.N_HID, L.N_IN)) * 0.2, "b1": rng.standard_normal(L.N_HID) * 0.1,
         "W2": rng.standard_normal((L.N_HID, L.N_HID)) * 0.1, "b2": rng.standard_normal(L.N_HID) * 0.1,
         "W3": rng.standard_normal((L.N_OUT, L.N_HID)) * 0.1, "b3": rng.standard_normal(L.N_OUT) * 0.1}
    return L.pack(d).astype(np.float32)


def _weight_mask():
    return L.pack({k: np.full(shape, k.startswith("W"), dtype=np.float64) for k, shape in L.SHAPES}).astype(bool)


def _bits(x32):
    return synth.to_bf16_bits(np.asarray(x32, dtype=np.float64)).astype(np.uint16)


def test_mlp_kernels_match_oracle(lrs):
    torch = _torch()
    P = int(lrs.lib.lrs_mlp_param_count())
    p32 = _random_params(0)
    assert P == p32.size
    mask = _weight_mask()
    rng = np.random.default_rng(1)
    B = 37                                               # ragged against the 256-thread blocks
    X = rng.uniform(-1.0, 1.0, (B, L.N_IN)).astype(np.float32)
    y = rng.integers(0, L.N_OUT, B).astype(np.int32)
    dev = "cuda"
    p = torch.from_numpy(p32.copy()).to(dev)
    w = torch.zeros(P, dtype=torch.int16, device=dev)
    lrs.mlp_init_bf16(p, w)
    wb = w.cpu().numpy().view(np.uint16)
    assert np.array_equal(wb[mask], _bits(p32[mask])) and not wb[~mask].any()

    Xd, yd = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
    logits = torch.empty((B, L.N_OUT), dtype=torch.float32, device=dev)
    lrs.mlp_forward(p, w, Xd, B, logits)
    grad = torch.zeros(P, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    lrs.mlp_loss_grad(p, w, Xd, yd, B, grad, loss)
    torch.cuda.synchronize()

    d = L.unpack(p32.astype(np.float64))
    z_o, _ = L.mlp_forward(d, X.astype(np.float64))
    loss_o, g_o = L.mlp_loss_grad(d, X.astype(np.float64), y)
    # FP32 accumulation of at most 128 products per sum: relative 2e-5 of the scale
    z = logits.cpu().numpy()
    assert np.max(np.abs(z - z_o)) <= 2e-5 * np.max(np.abs(z_o))
    assert abs(float(loss.item()) - loss_o) <= 2e-5 * loss_o
    g = L.unpack(grad.cpu().numpy().astype(np.float64))
    for k in g_o:
        scale = np.max(np.abs(g_o[k]))
        assert np.max(np.abs(g[k] - g_o[k])) <= 2e-5 * scale + 1e-9, k

    # two Adam steps against the restated update, then the refreshed BF16 weights
    m1 = torch.zeros(P, dtype=torch.float32, device=dev)
    m2 = torch.zeros(P, dtype=torch.float32, device=dev)
    po, m1o, m2o = p32.astype(np.float64), np.zeros(P), np.zeros(P)
    for step in (1, 2):
        lrs.mlp_loss_grad(p, w, Xd, yd, B, grad, loss)
        gh = grad.cpu().numpy().astype(np.float64)
        lrs.mlp_adam(p, w, grad, m1, m2, step, 1e-3)
        po, m1o, m2o = L.adam_step(po, gh, m1o, m2o, step, 1e-3)
        ph = p.cpu().numpy()
        assert np.max(np.abs(ph - po)) <= 1e-6 * np.max(np.abs(po)) + 1e-7
        po = ph.astype(np.float64)                       # continue from the device's FP32 state
        m1o, m2o = m1.cpu().numpy().astype(np.float64), m2.cpu().numpy().astype(np.float64)
    wb = w.cpu().numpy().view(np.uint16)
    assert np.array_equal(wb[mask], _bits(p.cpu().numpy()[mask]))


def _matrix(sp):
    return np.ascontiguousarray(recipe.matrix(sp), dtype=np.float32)


@pytest.mark.parametrize("spec", [
    dict(field="tanh", N=32, m=200, nfronts=3, nblobs=2, seed=901),
    dict(field="blob", N=64, m=333, nfronts=1, nblobs=12, seed=902),
    dict(field="heat", N=64, m=97, nfronts=1, nblobs=2, seed=903),
    dict(field="tanh", N=128, m=450, nfronts=2, nblobs=2, seed=904),
])
def test_basis_features_match_oracle(lrs, spec):
    torch = _torch()
    from paper_2105_01271_gb300 import learned
    A = _matrix(spec)
    m, N = A.shape[0], spec["N"]
    Ad = torch.from_numpy(A).cuda()
    bufs = learned.buffers(m, N, Ad.device)
    Q, ldq, r, l = learned.basis(lrs, Ad, m, N, 0, bufs, diag=True)
    x = learned.basis_features(lrs, m, N, bufs, r, l).cpu().numpy().ravel().astype(np.float64)
    xo = L.features(A, N)
    # the sizes are exact; the rank may differ by one at the stop threshold
    assert np.allclose(x[L.N_SIGMA:L.N_SIGMA + 2], xo[L.N_SIGMA:L.N_SIGMA + 2], atol=1e-6)
    ro = int(round(xo[-1] * min(m, l)))
    assert abs(r - ro) <= 1
    # log |R_ii|: close where they are clear of the clip at 1e-6
    clear = xo[:L.N_SIGMA] > -0.9
    assert np.max(np.abs(x[:L.N_SIGMA][clear] - xo[:L.N_SIGMA][clear]), initial=0.0) <= 1e-4
    assert np.all(x[:L.N_SIGMA][~clear] <= -0.85)


@pytest.fixture(scope="module")
def trained(lrs):
    if not os.path.exists(SET):
        pytest.skip("tests/golden/learned_set.npz not generated")
    from paper_2105_01271_gb300 import learned
    torch = _torch()
    d = np.load(SET)
    model = learned.Proposal(lrs, seed=0)
    Xd = torch.from_numpy(d["X_train"].astype(np.float32)).cuda()
    yd = torch.from_numpy(d["y_train"].astype(np.int32)).cuda()
    loss0 = float(model.loss_grad(Xd, yd)[0].item())       # the untrained network on the whole set
    hist = model.train(d["X_train"], d["y_train"], epochs=120, batch=128, lr=2e-3, seed=0)
    return model, [loss0] + hist, d


def test_training_on_gpu_reduces_loss_and_predicts(trained):
    model, hist, d = trained
    assert hist[-1] < 0.5 * hist[0], hist[::20]             # hist[0]: before the first step
    pred = model.predict(d["X_test"])
    y = d["y_test"]
    acc = float(np.mean(pred == y))
    # oracle-table cost: configurations tried until one passes, from the start
    E = d["err_test"]
    def tries(start, e):
        ok = np.nonzero(e[start:] <= TOL)[0]
        return (ok[0] + 1) if ok.size else len(e) - start
    adaptive = np.mean([tries(0, e) for e in E])
    learned_ = np.mean([tries(int(p), e) for p, e in zip(pred, E)])
    print(f"\nheld-out accuracy {acc:.3f}; tries per matrix: adaptive {adaptive:.2f}, learned {learned_:.2f}")
    assert acc >= 0.6
    assert learned_ < adaptive


def test_learned_start_beats_adaptive_enlargement(lrs, trained):
    """Held-out matrices, regenerated from the stored recipe: both variants
    reach the tolerance (checked on the device and, for the accepted
    configuration, in the oracle's table); the learned start tries fewer
    configurations and takes less time in total."""
    torch = _torch()
    from paper_2105_01271_gb300 import learned
    model, _, d = trained
    meta, E = d["meta_test"], d["err_test"]
    pick = np.random.default_rng(0).choice(len(meta), 40, replace=False)
    mats = []
    for i in pick:
        f, N, m, nf, nb, seed = (int(v) for v in meta[i])
        sp = dict(field=recipe.FIELDS[f], N=N, m=m, nfronts=nf, nblobs=nb, seed=seed)
        mats.append((i, N, m, torch.from_numpy(_matrix(sp)).cuda()))
    Nmax = max(N for _, N, _, _ in mats)
    mmax = max(m for _, _, m, _ in mats)
    bufs = learned.buffers(mmax, Nmax, "cuda")
    # warm-up: grow every workspace to its largest size once
    big = max(mats, key=lambda t: t[1] * t[1] * t[2])
    for _ in range(2):
        learned.decompose_to_tolerance(lrs, big[3], big[2], big[1], TOL, bufs, start=len(learned.CONFIGS) - 1)
        learned.decompose_to_tolerance(lrs, big[3], big[2], big[1], TOL, bufs, model=model)
    tot = {"adaptive": [0.0, 0], "learned": [0.0, 0]}
    for i, N, m, A in mats:
        for name, kw in (("adaptive", {}), ("learned", {"model": model})):
            run = learned.decompose_to_tolerance(lrs, A, m, N, TOL, bufs, **kw)
            tot[name][0] += run.seconds
            tot[name][1] += len(run.tried)
            err = run.tried[-1][1]
            if run.accepted < len(learned.CONFIGS) - 1:
                assert err <= TOL
                assert E[i][run.accepted] <= 2 * TOL, (i, run.accepted, E[i])
    print(f"\n40 held-out matrices: adaptive {tot['adaptive'][0] * 1e3:.1f} ms / {tot['adaptive'][1]} tries, "
          f"learned {tot['learned'][0] * 1e3:.1f} ms / {tot['learned'][1]} tries")
    assert tot["learned"][1] < tot["adaptive"][1]
    assert tot["learned"][0] < tot["adaptive"][0]
