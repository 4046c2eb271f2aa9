"""Benchmark: particles/s per CRKSPH + short-range-gravity step.

One step = one pass of the whole hot path on one batch of particles: first
half kick and drift, Morton keys, radix sort, permutation, leaves, leaf
hierarchy, leaf-pair lists, density, moments + corrections, hydro, gravity,
second half kick.  Workload: the 2 x 128^3 Gaussian-random-field box
(P(k) ~ k^-2, 0.3-cell rms displacement, ~270 gas neighbours), FP32-mixed
form, inputs resident in HBM (about 2.5 GB of state, far larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own independent box (weak
scaling, no collective on the data path); the barrier and the max over
ranks only bracket the timing.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s per CRKSPH+SR-gravity step, mixed vs FP64; serve p50/p99 ms"
UNIT = "particles/s"

# Algorithmic FP32 operations of one in-range pair, counted from the kernels'
# pair bodies in csrc/passes.cu with the paper's convention (Sec. VI-B: FMA =
# 2, add/mul = 1, sqrt/rsqrt/exp/reciprocal = 1).  Pairs outside the support
# (leaf-pair overlap) are not counted.
FLOP_PER_PAIR = {"density": 22, "moments": 125, "hydro": 183, "gravity": 41}
# GB300's FP64 rate (vector and tensor alike are far below its FP32 rate); a
# nominal figure, the denominator of the plain FP64 form's algorithmic rates.
FP64_NOMINAL_TFLOPS = 1.25

# DRAM bytes (read + write) per particle of one launch of each pass, from the
# one-pass ncu capture summarised in profiles/launches_gaussian_2x128.md
# (2x128^3 Gaussian field, leaf capacity 128; density = list bounds + fill
# with the density sum + kept counts).  They describe the kernels of the csrc/passes.cu with this
# SHA-256 only; for any other source the bench reports no traffic.
TRAFFIC_SOURCE_SHA256 = "695550b977dabc80776240b71028b5f1020dafab76880c791a1c4e7e33176915"
TRAFFIC_BYTES_PER_PARTICLE = {"gravity": 81.3, "hydro": 701.4, "moments": 690.8, "density": 1088.2}


def _traffic(kernel: str, particles: int, leaf_cap: int):
    import hashlib

    try:
        with open(os.path.join(ROOT, "paper_2510_03557_gb300", "csrc", "passes.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    if sha != TRAFFIC_SOURCE_SHA256 or leaf_cap != 128 or kernel not in TRAFFIC_BYTES_PER_PARTICLE:
        return None
    return round(TRAFFIC_BYTES_PER_PARTICLE[kernel] * particles)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, cmd=None):
        self.device = device
        self.proc = None
        self.cmd = cmd or ["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                           "--format=csv,noheader,nounits", "-lms", "100"]

    def __enter__(self):
        import select

        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return self
        # wait (at most 5 s) until the sampler runs, so that the timed region
        # is sampled from its start; the first record precedes it and is dropped
        ready, _, _ = select.select([self.proc.stdout], [], [], 5.0)
        if ready:
            self.proc.stdout.readline()
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            self.samples = []
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.samples = [l.split(",") for l in out.strip().splitlines() if l.count(",") >= 8]

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].strip().replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for k, name in enumerate(names):
            if any(s[5 + k].strip().lower() == "active" for s in self.samples):
                reasons.append(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def cpu_baseline(n: int = 80):
    """The CPU oracle as it stands, on a bounded sample of the same workload:
    one force evaluation plus one KDK step of a 2 x n^3 box from the same
    generator (same density, neighbour counts and h in spacing units)."""
    import oracle
    from paper_2510_03557_gb300 import workloads as wl

    oracle.build()
    box = wl.gaussian_field_box(n, seed=1)
    op = oracle.make_params(**box.params())
    t0 = time.perf_counter()
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op)
    t1 = time.perf_counter()
    oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, box.dt, 1,
               acc=ref["acc"], dudt=ref["dudt"])
    t2 = time.perf_counter()
    step_s = t2 - t1  # one KDK step = one force evaluation plus kicks and drift
    return {"value": box.n / step_s, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"one KDK step of a 2x{n}^3 box from the same generator (N={box.n}), "
                      f"force evaluation {t1 - t0:.2f} s"}


def serve_bench(crk, wl, args, stream):
    """The serving workload on a bounded sample: the first ``count`` requests
    of the 2,000-request stream (n log-uniform in [16, 128], 20 KDK steps at
    dt = 1e-3, FP32-mixed, 150 GB budget).  A closed-loop calibration batch
    fixes the saturated throughput; Poisson arrivals are then issued at 70% of
    it and the service reports each request's submit-to-completion latency.
    Beside it, sequential plain-FP64 solves (one handle per request, one box
    per launch) of a few of the same requests give the FP64 rate."""
    import concurrent.futures as cf

    count = args.serve_requests
    reqs = wl.serving_requests(2000)[:count]
    with cf.ThreadPoolExecutor(8) as ex:
        boxes = list(ex.map(lambda r: wl.gaussian_field_box(r[0], seed=r[1]), reqs))
    steps = 20
    svc = crk.crk_service_create(150 * 10**9, max_slots=64, precision=crk.CRK_MIXED,
                                 leaf_cap=args.serve_leaf_cap)

    def submit(b):
        return crk.crk_submit(svc, crk.box_physics(b), b.pos, b.vel, b.mass, b.u, b.h, b.species,
                              b.dt, steps)

    def collect(tickets, bs):
        return [crk.crk_poll(svc, t, b.n, -1) for t, b in zip(tickets, bs)]

    try:
        # calibration: a closed batch, everything submitted at once
        calib = boxes[:min(32, count)]
        t0 = time.perf_counter()
        collect([submit(b) for b in calib], calib)
        t_cal = time.perf_counter() - t0
        capacity = len(calib) / t_cal                       # requests/s when saturated
        rate = 0.7 * capacity
        arrivals = wl.poisson_arrivals(count, rate, seed=5)
        tickets = []
        t0 = time.perf_counter()
        for a, b in zip(arrivals, boxes):
            while time.perf_counter() - t0 < a:
                time.sleep(min(1e-3, max(0.0, a - (time.perf_counter() - t0))))
            tickets.append(submit(b))
        res = collect(tickets, boxes)
        wall = time.perf_counter() - t0
    finally:
        crk.crk_service_destroy(svc)
    lat = np.array([r["latency_ns"] for r in res]) / 1e6
    que = np.array([r["queue_ns"] for r in res]) / 1e6
    psteps = sum(b.n for b in boxes) * steps

    # sequential plain FP64: one request at a time, 2 steps each, on a few requests
    seq = boxes[:min(6, count)]
    t64 = 0.0
    p64 = 0
    for b in seq:
        s = crk.Sim(crk.box_physics(b), leaf_cap=args.leaf_cap, precision=crk.CRK_FP64, stream=stream)
        s.load(b)
        stream.synchronize()
        t1 = time.perf_counter()
        s.step(b.dt, 2)
        stream.synchronize()
        t64 += time.perf_counter() - t1
        p64 += b.n * 2
        s.close()
    return {"requests": count, "of": 2000, "steps_per_request": steps,
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "queue_p50_ms": round(float(np.percentile(que, 50)), 3),
            "value": psteps / wall, "unit": UNIT,
            "arrival_rate_per_s": round(rate, 3), "load": 0.7,
            "calibration": {"requests": len(calib), "seconds": round(t_cal, 3)},
            "fp64_sequential": {"value": p64 / t64, "unit": UNIT, "requests": len(seq),
                                "steps_per_request": 2}}


def _rel_l2(x, ref):
    d = np.linalg.norm(np.asarray(x) - np.asarray(ref))
    r = np.linalg.norm(np.asarray(ref))
    return float(d / r) if r > 0 else float(d)


def run_bins(args):
    """Hierarchical time steps on the clustered workload (2 x n^3, half in
    512 Plummer spheres, kNN h): one long step of 2^depth substeps of the
    initial Courant step d, against the fixed-step KDK that advances the same
    time at step d (what every particle needs when the deepest one needs d).
    The fixed-step time is measured over a few steps and scaled to 2^depth."""
    import torch

    from paper_2510_03557_gb300 import crk
    from paper_2510_03557_gb300 import workloads as wl

    torch.cuda.set_device(0)
    crk.lib()
    box = wl.clustered_box(args.n, seed=3)
    phys = crk.box_physics(box)
    stream = torch.cuda.Stream()
    depth = args.bin_depth
    d = box.dt
    dt_long = d * (1 << depth)
    s = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream)
    s.load(box)
    s.forces(counts=False)
    crk.crk_set_timing(s.handle, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clocks:
        e0.record(stream)
        counts = crk.crk_step_bins(s.handle, dt_long, depth, 1, args.bin_eta, args.bin_courant)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_bins = e0.elapsed_time(e1)
    tim = crk.crk_get_timings(s.handle)
    bins = crk.crk_get_bins(s.handle)
    s.close()
    f = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream)
    f.load(box)
    f.step(d, 1)
    k = max(1, min(args.steps, 1 << depth))
    torch.cuda.synchronize()
    e0.record(stream)
    f.step(d, k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fixed = e0.elapsed_time(e1) / k * (1 << depth)
    f.close()
    calls = max(tim["calls"], 1)
    line = {"metric": METRIC, "value": box.n * (1 << depth) / (ms_bins / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": 1, "ms_per_step": ms_bins, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"clustered 2x{args.n}^3, hierarchical steps: one long step of "
                                   f"2^{depth} substeps of d={d} (value: particles x substeps / time)",
                       "particles": box.n, "leaf_cap": args.leaf_cap, "depth": depth,
                       "eta": args.bin_eta, "courant": args.bin_courant},
            "bins": {"long_step_ms": round(ms_bins, 3), "fixed_step_ms_same_time": round(ms_fixed, 3),
                     "speedup": round(ms_fixed / ms_bins, 3),
                     "bin_histogram_after": np.bincount(bins, minlength=depth + 1).tolist(),
                     "active_per_substep": counts.tolist(),
                     "active_fraction": round(float(counts.sum()) / (box.n * (1 << depth)), 5),
                     "substep_breakdown_ms": {k2: round(tim[k2] / calls, 4) for k2 in
                                              ("tree_ms", "pairs_ms", "density_ms", "moments_ms",
                                               "hydro_ms", "gravity_ms", "kdk_ms")},
                     "fixed_steps_timed": k},
            "clocks": clocks.summary()}
    print(json.dumps(line))


def fp64_pass_rates(tim, pairs):
    """Per-phase times of the timed FP64 steps and each pair pass's
    algorithmic rate, also as a share of the nominal FP64 rate."""
    calls = max(tim["calls"], 1)
    rates = {k: pairs[k] * FLOP_PER_PAIR[k] / (tim[k + "_ms"] / calls / 1e3) / 1e12
             for k in ("density", "moments", "hydro", "gravity") if tim[k + "_ms"] > 0}
    return {"breakdown_ms": {k: round(tim[k] / calls, 3) for k in
                             ("tree_ms", "pairs_ms", "density_ms", "moments_ms", "hydro_ms",
                              "gravity_ms", "kdk_ms")},
            "pass_tflops": {k: round(v, 4) for k, v in rates.items()},
            "pass_of_fp64_peak": {k: round(v / FP64_NOMINAL_TFLOPS, 4) for k, v in rates.items()},
            "fp64_peak": {"value": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                          "source": "nominal GB300 FP64 rate, not measured"}}


def pair_census(tim, pairs, n_gas, n):
    """Evaluated / algorithmic pairs of the counted evaluation: candidate
    tests in lane slots (a warp tests its up to 32 targets against every staged
    candidate) per in-range pair, the hydro list entries per gather pair, and
    the share of walked list slots that hold an entry."""
    gather = pairs["density"]                 # ordered gather pairs, self included
    grav = pairs["gravity"] + n               # each target is also tested against itself
    r = lambda a, b: round(a / b, 3) if b else None
    return {"gravity": {"tested_slots": tim["tests_grav"], "target_slots": tim["tests_grav_target"],
                        "in_range": grav, "tested_per_in_range": r(tim["tests_grav"], grav),
                        "target_slots_per_in_range": r(tim["tests_grav_target"], grav)},
            "hydro_fill": {"tested_slots": tim["tests_hydro"], "list_entries": tim["list_entries"],
                           "gather_pairs": gather, "tested_per_entry": r(tim["tests_hydro"], tim["list_entries"]),
                           "entries_per_gather_pair": r(tim["list_entries"], gather)},
            "list_walk": {"slots": tim["list_slots"], "entries": tim["list_entries"],
                          "entry_share": r(tim["list_entries"], tim["list_slots"])},
            "note": "lane slots of one counted force evaluation; in-range gravity pairs include each "
                    "target's self test"}


def run_clustered(args):
    """Precision study on the clustered workload (2 x n^3, half uniform and
    half in 512 Plummer spheres, adaptive h): one force evaluation plus 5 KDK
    steps in the plain FP64 form and the FP32-mixed form, the mixed form's
    relative error per output against FP64, both forms' conserved-sum drift,
    and the FP64 form against the CPU oracle on a seeded sample of particles
    (the oracle only evaluates the sample and what it depends on)."""
    import torch

    import oracle
    from paper_2510_03557_gb300 import crk
    from paper_2510_03557_gb300 import workloads as wl

    torch.cuda.set_device(0)
    crk.lib()
    tg = time.perf_counter()
    box = wl.clustered_box(args.n, seed=3)
    t_gen = time.perf_counter() - tg
    phys = crk.box_physics(box)
    stream = torch.cuda.Stream()
    gas = box.species == wl.GAS
    runs = {}
    for name, prec in (("fp64", crk.CRK_FP64), ("mixed", crk.CRK_MIXED)):
        nsteps = box.nsteps if name == "mixed" or args.fp64_steps < 0 else args.fp64_steps
        s = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=prec, stream=stream)
        s.load(box)
        crk.crk_set_timing(s.handle, True)
        out = s.forces(counts=False)   # device phases timed by the library; the copy-out is not
        tf = crk.crk_get_timings(s.handle)
        force_ms = sum(tf[k] for k in ("tree_ms", "pairs_ms", "density_ms", "moments_ms", "hydro_ms",
                                       "gravity_ms", "kdk_ms"))
        mom0, e0, _ = crk.crk_get_sums(s.handle)
        crk.crk_set_timing(s.handle, True)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        failure = None
        if nsteps > 0:
            try:
                s.step(box.dt, nsteps)
            except crk.CrkError as e:
                failure = str(e)
        k1.record(stream)
        torch.cuda.synchronize()
        mom1, e1, nfl = crk.crk_get_sums(s.handle)
        tim = crk.crk_get_timings(s.handle)
        calls = max(tim["calls"], 1)
        pos, vel, u = s.state()
        pabs = float(np.sum(box.mass[:, None] * np.abs(vel)))
        runs[name] = dict(out=out, pos=pos, vel=vel, u=u, nsteps=nsteps, failure=failure,
                          force_ms=force_ms,
                          step_ms=k0.elapsed_time(k1) / nsteps if nsteps else None,
                          momentum_drift=float(np.linalg.norm(np.subtract(mom1, mom0))) / max(pabs, 1e-300),
                          energy_drift=(e1 - e0) / abs(e0), floor_events=nfl,
                          breakdown={k: round(tim[k] / calls, 3) for k in
                                     ("tree_ms", "pairs_ms", "density_ms", "moments_ms", "hydro_ms",
                                      "gravity_ms", "kdk_ms")},
                          leaves=int(tim["nleaves"]), leaf_pairs=[int(tim["pairs_hydro"]),
                                                                  int(tim["pairs_grav"])])
        if name == "mixed" and not args.no_extras:
            # friends-of-friends halos of the dark matter at b = 0.2 mean
            # spacings on the clustered state after the KDK steps
            torch.cuda.synchronize()
            t_f = time.perf_counter()
            grp, n_groups = crk.crk_fof(s.handle, 0.2 / args.n, 1, box.n)
            fof_ms = (time.perf_counter() - t_f) * 1e3
            _, sizes = np.unique(grp[grp >= 0], return_counts=True)
            runs[name]["fof"] = {"ms": round(fof_ms, 3), "groups": n_groups,
                                 "groups_20_or_more": int(np.sum(sizes >= 20)),
                                 "largest": int(sizes.max()) if len(sizes) else 0,
                                 "in_groups_20_or_more": round(float(sizes[sizes >= 20].sum()) / max(len(grp[grp >= 0]), 1), 4),
                                 "linking_length": 0.2 / args.n, "species": "dm",
                                 "note": "host wall time of crk_fof: tree build, links, labels, copy-out"}
            cnt = s.forces(counts=True)
            pc = {"density": int(cnt["nbr_count"][gas].sum()) + int(gas.sum()),
                  "gravity": int(cnt["grav_count"].sum())}
            runs[name]["census"] = pair_census(crk.crk_get_timings(s.handle), pc, int(gas.sum()), box.n)
        s.close()
    a, b = runs["mixed"], runs["fp64"]
    err = {"acc": _rel_l2(a["out"]["acc"], b["out"]["acc"]),
           "dudt": _rel_l2(a["out"]["dudt"][gas], b["out"]["dudt"][gas]),
           "A": _rel_l2(a["out"]["A"][gas], b["out"]["A"][gas]),
           "B": _rel_l2(a["out"]["B"][gas], b["out"]["B"][gas]),
           "gradA": _rel_l2(a["out"]["gradA"][gas], b["out"]["gradA"][gas]),
           "gradB": _rel_l2(a["out"]["gradB"][gas], b["out"]["gradB"][gas]),
           "rho": _rel_l2(a["out"]["rho"][gas], b["out"]["rho"][gas])}
    if a["nsteps"] == b["nsteps"] and not a["failure"] and not b["failure"]:
        tag = f"after_{a['nsteps']}_kdk"
        disp = lambda p: (p - box.pos + 0.5) % 1.0 - 0.5
        err.update({"displacement_" + tag: _rel_l2(disp(a["pos"]), disp(b["pos"])),
                    "vel_" + tag: _rel_l2(a["vel"], b["vel"]),
                    "u_" + tag: _rel_l2(a["u"][gas], b["u"][gas])})
    # FP64 form against the oracle on a seeded sample
    oracle.build()
    rng = np.random.default_rng(33)
    idx = np.concatenate([rng.choice(np.flatnonzero(gas), args.sample // 2, replace=False),
                          rng.choice(np.flatnonzero(~gas), args.sample // 2, replace=False)])
    op = oracle.make_params(**box.params())
    to = time.perf_counter()
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, sample=idx)
    t_or = time.perf_counter() - to
    gi = idx[gas[idx]]
    orc = {"acc": _rel_l2(b["out"]["acc"][idx], ref["acc"][idx]),
           "dudt": _rel_l2(b["out"]["dudt"][gi], ref["dudt"][gi]),
           "A": _rel_l2(b["out"]["A"][gi], ref["A"][gi]),
           "B": _rel_l2(b["out"]["B"][gi], ref["B"][gi])}
    orc_mixed = {"acc": _rel_l2(a["out"]["acc"][idx], ref["acc"][idx]),
                 "dudt": _rel_l2(a["out"]["dudt"][gi], ref["dudt"][gi]),
                 "A": _rel_l2(a["out"]["A"][gi], ref["A"][gi]),
                 "B": _rel_l2(a["out"]["B"][gi], ref["B"][gi])}
    fp64_rate = box.n / ((b["step_ms"] if b["step_ms"] else b["force_ms"]) / 1e3)
    line = {"metric": METRIC, "value": box.n / (a["step_ms"] / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": box.nsteps, "ms_per_step": a["step_ms"], "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"clustered 2x{args.n}^3 precision study (512 Plummer spheres, "
                                   f"kNN h), 1 force evaluation + {box.nsteps} KDK at dt={box.dt} "
                                   f"(FP64 form: {b['nsteps']} KDK)",
                       "particles": box.n, "leaf_cap": args.leaf_cap},
            "fp64_plain": {"value": fp64_rate, "unit": UNIT, "kdk_steps": b["nsteps"],
                           "rate_from": "KDK steps" if b["step_ms"] else "the force evaluation",
                           "ms_per_step": b["step_ms"], "force_ms": b["force_ms"],
                           "breakdown_ms": b["breakdown"], "momentum_drift": b["momentum_drift"],
                           "energy_drift": b["energy_drift"], "failure": b["failure"]},
            "mixed": {"ms_per_step": a["step_ms"], "force_ms": a["force_ms"], "failure": a["failure"],
                      "breakdown_ms": a["breakdown"], "momentum_drift": a["momentum_drift"],
                      "energy_drift": a["energy_drift"], "leaves": a["leaves"],
                      "leaf_pairs": a["leaf_pairs"]},
            "fof": a.get("fof"), "pair_census_after_kdk": a.get("census"),
            "mixed_vs_fp64_rel_l2": err,
            "fp64_vs_oracle_rel_l2": orc, "mixed_vs_oracle_rel_l2": orc_mixed,
            "oracle_sample": {"particles": int(len(idx)), "seconds": round(t_or, 2),
                              "cores": oracle.max_threads()},
            "setup_s": round(t_gen, 1)}
    print(json.dumps(line))


def run_batched(args):
    """The batched workload: 64 independent periodic boxes of 2 n^3 particles,
    n drawn (seed 2) from {16, 24, 32, 48, 64}, box b from the Gaussian-field
    generator with seed 1000 + b, all in one handle (one tree and one launch
    per pass for every box), FP32-mixed, leaf capacity chosen by the library's
    autotuner.  Beside it the plain FP64 form one box per handle, run one box
    after another, on the first 8 boxes."""
    import torch

    from paper_2510_03557_gb300 import crk
    from paper_2510_03557_gb300 import workloads as wl

    torch.cuda.set_device(0)
    crk.lib()
    boxes = wl.batched_boxes(64, seed=2)
    cat = wl.concat_boxes(boxes)
    N = int(cat["offsets"][-1])
    phys = [crk.box_physics(b) for b in boxes]
    dts = [b.dt for b in boxes]
    stream = torch.cuda.Stream()
    sim = crk.Sim(phys[0], leaf_cap=128, precision=crk.CRK_MIXED, stream=stream)
    crk.crk_load_boxes(sim.handle, [b.n for b in boxes], phys, cat["pos"], cat["vel"], cat["mass"],
                       cat["u"], cat["h"], cat["species"])
    sim.n = N
    best, tune_ms = crk.crk_autotune(sim.handle, (32, 64, 128))
    crk.crk_step_boxes(sim.handle, dts, args.warmup)
    crk.crk_set_timing(sim.handle, True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clocks:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        crk.crk_step_boxes(sim.handle, dts, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    tim = crk.crk_get_timings(sim.handle)
    calls = max(tim["calls"], 1)
    sim.close()
    t64 = 0.0
    p64 = 0
    for b in boxes[:8]:
        s = crk.Sim(crk.box_physics(b), leaf_cap=64, precision=crk.CRK_FP64, stream=stream)
        s.load(b)
        s.step(b.dt, 1)
        stream.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s.step(b.dt, 1)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 += f0.elapsed_time(f1) / 1e3
        p64 += b.n
        s.close()
    line = {"metric": METRIC, "value": N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched: 64 Gaussian-field boxes 2 n^3, n in {16,24,32,48,64} "
                                   "(seed 2), one handle, FP32-mixed, KDK dt=1e-3",
                       "particles": N, "boxes": len(boxes), "leaf_cap": best},
            "autotune_ms": {str(k): round(v, 3) for k, v in tune_ms.items()},
            "breakdown_ms": {k: round(tim[k] / calls, 4) for k in
                             ("tree_ms", "pairs_ms", "density_ms", "moments_ms", "hydro_ms",
                              "gravity_ms", "kdk_ms")},
            "gpu_launches_per_step": int(tim["launches"]) // max(args.steps, 1),
            "fp64_one_box_per_launch": {"value": p64 / t64, "unit": UNIT, "boxes": 8, "steps": 1},
            "clocks": clocks.summary()}
    print(json.dumps(line))


def headline_config(args, world: int) -> dict:
    """The headline workload's config: the 2 x n^3 Gaussian-field box of the
    generator (dt 1e-3), as both arms report it."""
    n = 2 * args.n ** 3
    return {"workload": f"gaussian-field 2x{args.n}^3, FP32-mixed, KDK dt=0.001",
            "particles": n, "leaf_cap": args.leaf_cap, "rebuild_every": args.rebuild_every,
            "parallelism": f"replicas{world}",
            "l2": f"inputs larger than L2 (~{n * 600 / 1e9:.1f} GB resident state)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline(40)
    for _ in range(args.steps):
        cb = cpu_baseline(40)
        steps.append(cb["value"])
    value = statistics.median(steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": headline_config(args, args.gpus),
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bin-depth", type=int, default=5, help="bins workload: substeps 2^depth")
    ap.add_argument("--bin-eta", type=float, default=0.025)
    ap.add_argument("--bin-courant", type=float, default=0.25)
    ap.add_argument("--workload", default="gaussian", choices=["gaussian", "clustered", "batched", "bins"],
                    help="clustered: the precision study; batched: 64 boxes in one handle "
                         "(each prints its own JSON line)")
    ap.add_argument("--sample", type=int, default=64, help="oracle sample of the precision study")
    ap.add_argument("--n", type=int, default=128, help="lattice size per species (2 n^3 particles)")
    ap.add_argument("--leaf-cap", type=int, default=128)
    ap.add_argument("--rebuild-every", type=int, default=1,
                    help="sort into new leaves every this many steps (boxes grow in between)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="KDK steps of the FP64 form (precision study: -1 = as many as the mixed form)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FOF and long-range mesh legs")
    ap.add_argument("--serve-requests", type=int, default=192,
                    help="requests of the serving stream to run (0: skip)")
    ap.add_argument("--serve-leaf-cap", type=int, default=64)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "clustered":
        run_clustered(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "bins":
        run_bins(args)
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2510_03557_gb300 import crk
    from paper_2510_03557_gb300 import replicas
    from paper_2510_03557_gb300 import workloads as wl

    def max_over_ranks(v: float) -> float:
        return replicas.max_over_ranks(v, dist, "cuda")

    crk.lib()
    box = wl.gaussian_field_box(args.n, seed=1)
    N = box.n
    dt = box.dt
    phys = crk.box_physics(box)
    stream = torch.cuda.Stream()

    # ---------------- mixed form, device-resident (the headline value)
    sim = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream,
                  rebuild_every=args.rebuild_every)
    sim.load(box)
    counts = sim.forces(counts=True)      # untimed: the true pair counts for the roofline
    gas = box.species == wl.GAS
    pairs = {"density": int(counts["nbr_count"][gas].sum()) + int(gas.sum()),
             "moments": int(counts["nbr_count"][gas].sum()) + int(gas.sum()),
             "hydro": int(counts["nbr_count"][gas].sum()),
             "gravity": int(counts["grav_count"].sum())}
    census = pair_census(crk.crk_get_timings(sim.handle), pairs, int(gas.sum()), N)
    for _ in range(args.warmup):
        sim.step(dt, 1)
    crk.crk_set_timing(sim.handle, True)
    barrier()
    with ClockSampler(local) as clocks:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # every rank steps its own box: all ranks' particles over the slowest rank's time
    value, t_max = replicas.job_throughput(N * args.steps, ms, dist, "cuda")
    tim = crk.crk_get_timings(sim.handle)
    per_pass_ms = {"density": tim["density_ms"], "moments": tim["moments_ms"],
                   "hydro": tim["hydro_ms"], "gravity": tim["gravity_ms"]}
    calls = max(tim["calls"], 1)
    dom = max(per_pass_ms, key=per_pass_ms.get)
    dom_ms = per_pass_ms[dom] / calls
    clk = clocks.summary()
    peaks, peak_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_max)
    achieved = pairs[dom] * FLOP_PER_PAIR[dom] / (dom_ms / 1e3) / 1e12
    pass_tflops = {k: pairs[k] * FLOP_PER_PAIR[k] / (per_pass_ms[k] / calls / 1e3) / 1e12
                   for k in per_pass_ms}
    breakdown = {k: round(v / calls, 4) for k, v in
                 (("tree_ms", tim["tree_ms"]), ("pairs_ms", tim["pairs_ms"]),
                  ("density_ms", tim["density_ms"]), ("moments_ms", tim["moments_ms"]),
                  ("hydro_ms", tim["hydro_ms"]), ("gravity_ms", tim["gravity_ms"]),
                  ("kdk_ms", tim["kdk_ms"]))}
    launches = int(tim["launches"])
    fof = mesh = None
    if not args.no_extras:
        # friends-of-friends groups of the dark matter at b = 0.2 mean spacings
        # (the call sorts a new tree for the current state, then links)
        torch.cuda.synchronize()
        t_f = time.perf_counter()
        _, n_groups = crk.crk_fof(sim.handle, 0.2 / args.n, 1, N)
        fof = {"ms": round((time.perf_counter() - t_f) * 1e3, 3), "groups": n_groups,
               "linking_length": 0.2 / args.n, "species": "dm",
               "note": "host wall time of crk_fof: tree build, links, labels, copy-out"}
    sim.close()

    if not args.no_extras:
        # the same KDK step with the long-range mesh (FP64 PM, n^3 cells)
        smesh = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream,
                        rebuild_every=args.rebuild_every, pm_grid=args.n)
        smesh.load(box)
        smesh.step(dt, 2)
        crk.crk_set_timing(smesh.handle, True)
        smesh.step(dt, 3)
        tmesh = crk.crk_get_timings(smesh.handle)
        mcalls = max(tmesh["calls"], 1)
        mesh = {"pm_grid": args.n, "pm_ms": round(tmesh["pm_ms"] / mcalls, 4),
                "step_ms": round(tmesh["total_ms"] / mcalls, 4),
                "note": "per KDK step, CUDA events on the handle's stream: deposit, cuFFT forward, "
                        "Green's function, 3 cuFFT inverse, gather (FP64)"}
        smesh.close()

    # ---------------- FP64 plain form on the same box
    fp64 = None
    if args.fp64_steps > 0:
        s64 = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=crk.CRK_FP64, stream=stream)
        s64.load(box)
        s64.step(dt, 1)
        crk.crk_set_timing(s64.handle, True)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.step(dt, args.fp64_steps)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = max_over_ranks(f0.elapsed_time(f1))
        fp64 = {"value": world * N * args.fp64_steps / (t64 / 1e3), "unit": UNIT,
                "ms_per_step": t64 / args.fp64_steps, "steps": args.fp64_steps, "dtype": "f64"}
        # the same pair sets as the mixed form (both decide them in FP64)
        fp64.update(fp64_pass_rates(crk.crk_get_timings(s64.handle), pairs))
        s64.close()

    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        se = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream)
        se.load(box)
        se.step(dt, 1)
        pin = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
        hp, hv, hu = pin((N, 3)), pin((N, 3)), pin(N)
        crk.crk_get_state(se.handle, hp, hv, hu)
        k_e2e = max(2, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(k_e2e):
            crk.crk_set_state(se.handle, hp, hv, hu)     # H2D of the step's inputs
            crk.crk_step(se.handle, dt, 1)
            crk.crk_get_state(se.handle, hp, hv, hu)     # D2H of the step's result
        g1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        te = max_over_ranks(max(g0.elapsed_time(g1), wall * 1e3))
        e2e = {"value": world * N * k_e2e / (te / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(hp.nbytes + hv.nbytes + hu.nbytes),
               "d2h_bytes_per_step": int(hp.nbytes + hv.nbytes + hu.nbytes), "steps": k_e2e}
        se.close()

    serving = None
    if args.serve_requests > 0:
        serving = serve_bench(crk, wl, args, stream)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": headline_config(args, world),
            "roofline": {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3),
                         "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                         "traffic": _traffic(dom, N, args.leaf_cap),
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                                           "2x128^3 capture (profiles/launches_gaussian_2x128.md), "
                                           "scaled by particles",
                         "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                        f"({peak_kind} sm_max_mhz)"},
            "pass_tflops": {k: round(v, 3) for k, v in pass_tflops.items()},
            "pairs_per_step": pairs,
            "pair_census": census,
            "leaves": int(tim["nleaves"]), "leaf_pairs": {"hydro": int(tim["pairs_hydro"]),
                                                          "gravity": int(tim["pairs_grav"])},
            "breakdown_ms": breakdown,
            "fp64_plain": fp64,
            "fof": fof,
            "long_range_mesh": mesh,
            "serving": serving,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cb,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
