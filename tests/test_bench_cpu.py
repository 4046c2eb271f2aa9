"""Host logic of ``bench.py`` (no GPU): the FP32 peak, the clock-record
summary, the pair census ratios and the traffic table's source guard."""
import hashlib
import os

import pytest

import bench


def test_fp32_peak_is_sms_times_lanes_times_fma_times_clock():
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.fp32_peak_tflops(1000.0) == pytest.approx(38.912)
    assert bench.fp32_peak_tflops(1000.0, sms=76) == pytest.approx(38.912 / 2)


def test_algorithmic_pairs_count_forces_per_unordered_pair():
    """Density and moments per ordered gather pair with self; hydro per
    unordered union pair (from the list entries, which include each gas
    target itself); gravity per unordered pair."""
    import numpy as np

    gas = np.array([True, True, False, True])
    counts = {"nbr_count": np.array([4, 6, 0, 2]), "grav_count": np.array([10, 12, 8, 6])}
    p = bench.algorithmic_pairs(counts, gas, list_entries=3 + 20)
    assert p == {"density": 15, "moments": 15, "hydro": 10, "gravity": 18}
    # without list entries the gather sets stand in for the union sets
    assert bench.algorithmic_pairs(counts, gas)["hydro"] == 6


def _sampler(rows):
    s = bench.ClockSampler(0)
    s.samples = [r.split(",") for r in rows]
    return s


def test_clock_summary_median_max_and_reasons():
    idle = "Not Active"
    rows = [f"0, {mhz}, 2070, 900.0, 0x0, {idle}, {idle}, {idle}, {cap}"
            for mhz, cap in ((2070, idle), (2055, "Active"), (2070, idle))]
    out = _sampler(rows).summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    hot = _sampler([f"0, 1500, 2070, 1400.0, 0x0, Active, {idle}, Active, {idle}"]).summary()
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples_says_so():
    s = bench.ClockSampler(0)
    s.samples = []
    assert s.summary()["reasons"] == ["unsampled"]


def test_pair_census_ratios():
    tim = {"tests_grav": 3200, "tests_grav_target": 2000, "tests_hydro": 640, "list_entries": 200,
           "list_slots": 320}
    c = bench.pair_census(tim, 190, 300, n=20)
    # each of the 20 targets is also tested against itself
    assert c["gravity"]["in_range"] == 320
    assert c["gravity"]["tested_per_in_range"] == 10.0
    assert c["gravity"]["target_slots_per_in_range"] == 6.25
    assert c["hydro_fill"]["tested_per_entry"] == 3.2
    assert c["hydro_fill"]["entries_per_gather_pair"] == pytest.approx(1.053, abs=1e-3)
    assert c["list_walk"]["entry_share"] == 0.625
    empty = bench.pair_census({k: 0 for k in tim}, 0, 0, 0)
    assert empty["gravity"]["tested_per_in_range"] is None


def test_traffic_only_for_the_captured_source_and_capacity():
    assert bench._traffic("gravity", 1000, 64) is None
    assert bench._traffic("tree", 1000, 128) is None
    path = os.path.join(bench.ROOT, "paper_2510_03557_gb300", "csrc", "passes.cu")
    with open(path, "rb") as f:
        same = hashlib.sha256(f.read()).hexdigest() == bench.TRAFFIC_SOURCE_SHA256
    t = bench._traffic("gravity_pairs_once", 1000, 128)
    if same:
        assert t == round(bench.TRAFFIC_BYTES_PER_PARTICLE["gravity_pairs_once"] * 1000)
    else:
        assert t is None
    assert bench._traffic("gravity_gather", 1000, 128) is None   # no capture of that kernel's step form


def test_fp64_pass_rates():
    tim = {"calls": 2, "tree_ms": 2.0, "pairs_ms": 4.0, "density_ms": 20.0, "moments_ms": 0.0,
           "hydro_ms": 200.0, "gravity_ms": 100.0, "kdk_ms": 1.0}
    pairs = {"density": 1_000_000, "moments": 1_000_000, "hydro": 2_000_000, "gravity": 5_000_000}
    r = bench.fp64_pass_rates(tim, pairs, 1.1, "probe")
    assert r["breakdown_ms"]["hydro_ms"] == 100.0 and r["breakdown_ms"]["tree_ms"] == 1.0
    # 2e6 pairs x 183 flop in 0.1 s
    assert r["pass_tflops"]["hydro"] == pytest.approx(2e6 * 183 / 0.1 / 1e12, abs=1e-4)  # 4 decimals
    assert "moments" not in r["pass_tflops"]          # untimed phase: no rate
    assert r["pass_of_fp64_peak"]["gravity"] == pytest.approx(5e6 * 41 / 0.05 / 1e12 / 1.1, abs=1e-4)
    assert r["fp64_peak"] == {"value": 1.1, "unit": "TFLOP/s", "source": "probe"}


def test_reference_arm_line(tmp_path):
    """``--impl reference`` times the oracle on a bounded sample and reports
    the headline arm's config, metric and unit, with zero transfer bytes."""
    import argparse
    import json
    import subprocess
    import sys

    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--n", "32", "--ref-sample", "64"],
                         capture_output=True, text=True, check=True,
                         cwd=bench.ROOT, timeout=600).stdout.strip().splitlines()
    line = json.loads(out[-1])
    args = argparse.Namespace(n=32, nsphere=512, leaf_cap=128, rebuild_every=1, autotune=True)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"] == bench.headline_config(args, 1)
    assert "clustered 2x32^3" in line["config"]["workload"]
    assert line["higher_is_better"] is True and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and "64 seeded random particles" in cb["sample"]
    assert cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_clock_sampler_records_the_region_after_its_first_sample():
    """The sampler waits for its first record, drops it, and keeps what the
    sampling command prints while the region runs (a stand-in command here)."""
    import sys
    import time

    line = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    prog = ("import sys, time\n"
            "print('0, 1, 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active', flush=True)\n"
            "time.sleep(0.3)\n"
            f"for _ in range(3): print({line!r}, flush=True); time.sleep(0.05)\n"
            "time.sleep(30)\n")
    with bench.ClockSampler(0, cmd=[sys.executable, "-c", prog]) as s:
        time.sleep(0.8)
    out = s.summary()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["reasons"] == []


def test_clock_sampler_without_the_tool():
    with bench.ClockSampler(0, cmd=["/nonexistent/sampler"]) as s:
        pass
    assert s.summary()["reasons"] == ["unsampled"]
