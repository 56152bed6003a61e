"""Writes tests/golden/learned_set.npz: features and labels of the learned
sketch proposal for seeded synthetic matrices, computed by the FP64 oracle
only (oracle.learned) from synth's generators.

    python tests/golden/make_learned_set.py [--train 20000] [--test 1000] [--procs N]

Matrices: 2-D fields on N x N grids, N in {32, 64, 128}, m in [64, 512]
snapshots, FP32 storage: the heat field (16 modes; 20%), advected blobs (2-16
blobs; 40%) and traveling tanh fronts (1-4 fronts, sharpness 10-200; 40%).
meta columns: field, N, m, fronts, blobs, seed.  Train and test draw
from disjoint seeds.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FIELDS = synth.LEARNED_FIELDS
specs = synth.learned_specs
matrix = synth.learned_matrix


def one(sp):
    import oracle.learned as L
    A = matrix(sp).astype(np.float64)
    y, errs = L.label(A, sp["N"])
    return L.features(A, sp["N"]), y, np.array(errs)


def build(count, seed, procs):
    sps = specs(count, seed)
    res = []
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        for r in pool.imap(one, sps, chunksize=2):
            res.append(r)
            if len(res) % 50 == 0:
                print(f"  {len(res)}/{len(sps)}  {time.time() - t0:.0f} s", flush=True)
    X = np.stack([r[0] for r in res])
    y = np.array([r[1] for r in res], dtype=np.int32)
    E = np.stack([r[2] for r in res])
    meta = np.array([[FIELDS.index(s["field"]), s["N"], s["m"], s["nfronts"], s["nblobs"], s["seed"]] for s in sps],
                    dtype=np.int64)
    return X, y, E, meta


def main():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")       # one BLAS thread per worker (inherited by the spawned pool)
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=1000)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--out", default=os.path.join(HERE, "learned_set.npz"))
    a = ap.parse_args()
    Xtr, ytr, Etr, Mtr = build(a.train, 7, a.procs)
    Xte, yte, Ete, Mte = build(a.test, 8, a.procs)
    np.savez_compressed(a.out, X_train=Xtr, y_train=ytr, err_train=Etr, meta_train=Mtr,
                        X_test=Xte, y_test=yte, err_test=Ete, meta_test=Mte)
    print("labels (train):", np.bincount(ytr, minlength=6), " (test):", np.bincount(yte, minlength=6))


if __name__ == "__main__":
    main()
