"""The stored oracle results of the headline workload
(tests/golden/blob2d_m2000_512x512_f32.json, written by
tests/golden/make_blob2d_full.py from oracle/ and synth/ only) describe the
workload bench.py runs, and hang together as the paper's definitions require:

  * the workload's name, sizes, rank k, C-PWR passes q and rank cut rtol are
    the bench workload's;
  * r singular values of B, non-increasing, S_k their first k;
  * the error estimate is sqrt(sum_{i > k} s_i(B)^2 / ||A_f||_F^2) (the
    energy of B beyond rank k, Alg. 2) and, U_k S_k V_k^T being the
    projection U_k U_k^T A_f, a lower bound of the stored true error eps;
  * J holds k distinct snapshot indices; on the clear-gap variant every pivot
    margin is clear (> 1e-2) and J is the spiked snapshots in the order of
    their amplitudes (Alg. 4 takes the largest remaining row first).
"""
import json
import math
import os

import numpy as np

import bench
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "blob2d_m2000_512x512_f32.json")))


def test_golden_is_the_bench_workload():
    w, rtol = bench.workload_params(GOLD["workload"])
    assert w is synth.WORKLOADS[GOLD["workload"]]
    assert (GOLD["m"], GOLD["n"], GOLD["k"], GOLD["q"]) == (w.m, w.n, w.k, w.q)
    assert GOLD["rtol"] == rtol


def _check_field(f, k, m):
    sB = np.array(f["sB"])
    assert f["r"] == sB.size and f["r"] >= k
    assert np.all(np.diff(sB) <= 0)
    assert np.array_equal(np.array(f["S"]), sB[:k])
    tail = math.fsum(float(s) ** 2 for s in sB[k:])
    assert abs(f["err_est_svd"] - math.sqrt(tail / f["fro2"])) <= 1e-12 * f["err_est_svd"]
    assert f["err_est_svd"] <= f["eps"] * (1 + 1e-12)
    J = np.array(f["J"])
    assert J.size == k and np.unique(J).size == k and J.min() >= 0 and J.max() < m
    assert len(f["gaps"]) == k


def test_blob_results_are_consistent():
    _check_field(GOLD["blob"], GOLD["k"], GOLD["m"])


def test_spiked_results_are_consistent():
    f = GOLD["spiked"]
    _check_field(f, GOLD["k"], GOLD["m"])
    assert min(f["gaps"]) > 1e-2
    assert f["J"] == f["spiked_rows"][:GOLD["k"]]
