"""Writes tests/golden/blob2d_m2000_512x512_f32.json: the FP64 oracle's results
on the headline workload (2000 x 512^2 FP32 blob field, full weighting s = 16
onto 32^2, one C-PWR pass on the 4x injection subsample, k = 50, rtol 1e-6)
and on its clear-pivot-gap variant (synth.spiked_blob_field, 50 spiked
snapshots), computed only by oracle/ from synth's generators.

    python tests/golden/make_blob2d_full.py

Stored per field: the SVD path (Alg. 7 with re-orthonormalisation, then
Alg. 2): the basis rank r, every singular value of B = Q^T A_f, S_k, the
error estimate, the relative Frobenius error eps of U_k S_k V_k^T (Sec. 6),
||A_f||_F^2 and the RMS and maximum of the entries of |Q|^T |A_f| (the scale
of the product error terms); the ID path (Alg. 7 without
re-orthonormalisation, then Alg. 4): J, the pivot margins of the k CPQR
steps, the coarse-ID error estimate and the relative error of P A_f(J,:).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "blob2d_m2000_512x512_f32.json")
# clear-pivot-gap variant: 50 spiked snapshots, amplitudes 1000 * 0.97^j
SPIKE = dict(nspikes=50, ratio=0.97, amp0=1000.0)


def abs_product_scale(A, Q, col_block=1 << 15):
    """RMS and max entry of |Q|^T |A| (r x n), streamed over column slabs."""
    aq = np.abs(Q)
    ss, mx, cnt = 0.0, 0.0, 0
    for c0 in range(0, A.shape[1], col_block):
        P = aq.T @ np.abs(A[:, c0:c0 + col_block])
        ss += float(np.sum(P * P))
        mx = max(mx, float(P.max()))
        cnt += P.size
    return float(np.sqrt(ss / cnt)), mx


def run(A, w):
    t0 = time.time()
    o = oracle.svd_path(A, w.grid, w.k, q=w.q, gram_grid=w.gram, rtol=1e-6)
    eps = oracle.rel_fro_error(A, o["U"], o["S"], o["V"])
    rms, mx = abs_product_scale(A, o["Q"])
    d = oracle.id_path(A, w.grid, w.k, q=w.q, gram_grid=w.gram, rtol=1e-6)
    gaps = []
    oracle.row_id(d["G"], w.k, gaps)
    id_err = oracle.id_rel_error(A, d["J"], d["P"])
    print(f"  oracle {time.time() - t0:.1f} s: r {o['r']}, eps {eps:.6e}, id err {id_err:.6e}, "
          f"min gap {min(gaps):.3e}", flush=True)
    return {"r": int(o["r"]), "sB": [float(x) for x in o["sB"]], "S": [float(x) for x in o["S"]],
            "err_est_svd": float(o["err_est"]), "eps": float(eps), "fro2": float(o["fro2"]),
            "absQA_rms": rms, "absQA_max": mx,
            "J": [int(x) for x in d["J"]], "gaps": [float(x) for x in gaps[:w.k]],
            "err_est_id": float(d["err_est"]), "id_err": float(id_err)}


def main():
    w = synth.WORKLOADS["blob2d_m2000_512x512_f32"]
    out = {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "q": w.q, "rtol": 1e-6,
           "source": "FP64 oracle (oracle/), written by tests/golden/make_blob2d_full.py"}
    print("blob field", flush=True)
    A = synth.make_workload(w).astype(np.float64)
    out["blob"] = run(A, w)
    del A
    print("spiked blob field", flush=True)
    A, rows = synth.spiked_blob_field(w.m, w.N, w.params["nblobs"], w.params["seed"], s=w.grid.s[0],
                                      kappa=w.params["kappa"], **SPIKE)
    out["spiked"] = run(A.astype(np.float64), w)
    out["spiked"]["params"] = SPIKE
    out["spiked"]["spiked_rows"] = [int(x) for x in rows]
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
