"""Host logic of bench.py that needs no GPU: the parity object's tolerance
rule and counts, the traffic constants' guard, and the reference arm's
JSON line."""

import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _result(c, mu_rc, mu_rp):
    return {"c": c, "mu_r_cost": mu_rc, "mu_r_prob": mu_rp, "r_cost": mu_rc, "r_prob": mu_rp, "gap_states": 10,
            "gap_mismatch": 0, "mismatch_max_gap": 0.0, "mismatch_max_loss": 0.0}


def test_parity_tolerance_scales_with_eps_and_counts_pairs():
    nI, nJ, K = 2, 3, 2
    W = np.full((K, nI + nJ), 0.2)
    full = {"c": np.zeros((K, nI, nJ)), "r_cost": np.zeros((K, nI, nJ)), "r_prob": np.zeros((K, nI, nJ))}
    full["c"][1, 1, 2] = 5e-6  # engine c off by 5e-6 on one pair
    results = [(p, k, _result(0.0, 0.0, 0.0)) for p in range(nI * nJ) for k in range(K)]
    at_1e8 = bench._parity(results, full, W, nI, nJ, 1e-8)
    assert at_1e8["tolerance"] == 1e-6 and at_1e8["pairs_over_tolerance"]["c"] == 1
    assert at_1e8["worst_c"] == {"agent": 1, "task": 2, "weight": 1, "engine_minus_oracle": 5e-6}
    at_1e6 = bench._parity(results, full, W, nI, nJ, 1e-6)
    assert abs(at_1e6["tolerance"] - 1e-4) < 1e-15 and at_1e6["pairs_over_tolerance"]["c"] == 0
    assert at_1e6["pairs"] == nI * nJ * K


def test_traffic_constants_follow_the_profiled_source():
    prof = bench.TRAFFIC_PROFILES[("grid32-10x20-K16", "fp32")]
    t = bench._traffic("grid32-10x20-K16", "fp32", prof["variant"], prof["alg_bytes"])
    if bench._sweep_source_hash() == prof["sweep_source"]:
        assert t == prof["dram_bytes"]
    else:
        assert t is None
    assert bench._traffic("grid32-10x20-K16", "fp32", prof["variant"] + 1, 1.0) is None


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-budget", "0.5"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
