"""Host-side bookkeeping of bench.py (no GPU): kernel launch counts, per-stage rooflines."""
import math

import bench


C2_INFO = dict(P=24, Mt=96, M3=64, n0=288, nI=192, n_I_modes=4, cells=[20, 20, 20])
C3_INFO = dict(P=24, Mt=160, M3=1024, n0=480, nI=320, n_I_modes=32, cells=[33, 33, 266])
PEAKS = {"hbm_gbs": 6794.8, "sm_max_mhz": 2070.0}
FP32 = 152 * 128 * 2 * 2070e6 / 1e12
ALU = {"sms": 152, "sm_max_mhz": 2070.0, "fp32_derived": FP32, "fp32_measured": 74.0,
       "fp64_derived": 152 * 2 * 2 * 2070e6 / 1e12, "fp64_measured": 1.2}


def test_kernels_per_eval_matches_the_launch_lists():
    # ncu launch lists: 190 launches for 10 evaluations at N = 10^5 (pack, scan, scatter, spread, z pass,
    # 3 x 3 slab-class passes, z pass, gather, real space, finalize, energy); at N = 10^6 in [1,1,8]
    # the 290 037 real-space cells add the three-kernel multi-block scan
    assert bench.kernels_per_eval(C2_INFO, True) == 19
    assert bench.kernels_per_eval(C3_INFO, True) == 22
    assert bench.kernels_per_eval(C2_INFO, False) == 18
    # no mode in the set I: one slab class less
    assert bench.kernels_per_eval(dict(C2_INFO, n_I_modes=0), True) == 16


def test_stage_rooflines_report_each_stage_against_its_bound():
    ms = {"pack": 0.8, "spread": 5.0, "fourier": 0.8, "gather": 4.0, "real": 9.0, "final": 0.1}
    n, P = 100_000, 24
    pairs = n * 1e5 * 4.0 / 3.0 * math.pi * 0.15 ** 3
    r = bench.stage_rooflines(ms, 10, C2_INFO, n, "mixed", PEAKS, P, pairs, bench.alu_peak_for(ALU, "mixed")[0])
    assert set(r) == set(ms)
    fp32 = FP32
    for k in ("spread", "gather", "real"):
        assert r[k]["bound"] == "alu" and r[k]["unit"] == "TFLOP/s"
        assert r[k]["peak"] == fp32
    for k in ("pack", "fourier", "final"):
        assert r[k]["bound"] == "hbm" and r[k]["unit"] == "GB/s" and r[k]["peak"] == PEAKS["hbm_gbs"]
    for v in r.values():
        assert v["frac"] == v["achieved"] / v["peak"]
    # spread: 2 P^3 flop per particle over its time per evaluation
    assert math.isclose(r["spread"]["achieved"], n * 2 * P ** 3 / 0.5e-3 / 1e12)
    assert math.isclose(r["real"]["achieved"], pairs * 40 / 0.9e-3 / 1e12)
    # FP64 runs against the FP64 rate, and its Fourier passes move twice the FP32 grid bytes
    r64 = bench.stage_rooflines(ms, 10, C2_INFO, n, "fp64", PEAKS, P, pairs, bench.alu_peak_for(ALU, "fp64")[0])
    assert r64["spread"]["peak"] == ALU["fp64_derived"]
    assert bench.fourier_bytes(C2_INFO, 8) > bench.fourier_bytes(C2_INFO, 4)


def test_roofline_picks_the_dominant_stage():
    ms = {"pack": 0.8, "spread": 5.0, "fourier": 4.0, "gather": 4.0, "real": 14.0, "final": 0.1}
    rf = bench.roofline(ms, 10, C2_INFO, 100_000, "mixed", PEAKS, ALU, 1.26e8, "c2")
    assert rf["kernel"] == "k_real" and rf["bound"] == "alu"
    # the line's fraction is the work over the stage time over the unit-count peak
    assert math.isclose(rf["frac"], 1.26e8 * 40 / 1.4e-3 / 1e12 / FP32)
    assert "FMA-loop measured 74.00" in rf["peak_source"]
    ms["spread"] = 20.0
    rf = bench.roofline(ms, 10, C2_INFO, 100_000, "mixed", PEAKS, ALU, 1.26e8, "c2")
    assert rf["kernel"] == "k_spread"


def test_pair_count_matches_brute_force():
    """The roofline's pair count: every ordered pair with 0 < r <= rc over the z images, as a
    direct double loop finds it (short period, rc > L3/2, so several images of one pair count)."""
    import numpy as np
    rng = np.random.default_rng(7)
    L = (1.0, 1.0, 0.25)
    x = rng.random((300, 3)) * np.array(L)
    rc = 0.2
    brute = 0
    for a in range(len(x)):
        for img in range(-2, 3):
            d = x[a] - x - np.array([0.0, 0.0, img * L[2]])
            r = np.sqrt(np.sum(d * d, axis=1))
            brute += int(np.sum((r > 0) & (r <= rc)))
    assert bench.count_pairs(x, L, rc) == brute


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON line with the keys of
    the benchmark contract, its cpu_baseline and an e2e object without host-device copies."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "c1",
                          "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]
