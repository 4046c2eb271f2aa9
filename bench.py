"""Benchmark: particles/s per CRKSPH + short-range-gravity step.

One step = one pass of the whole hot path on one batch of particles: first
half kick and drift, Morton keys, radix sort, permutation, leaves, leaf
hierarchy, leaf-pair lists, density, moments + corrections, hydro, gravity,
second half kick.  Headline workload: the clustered 2 x 256^3 box (33.5 M
particles; per species half uniform, half in 512 Plummer spheres of scale
radius 0.002, adaptive h from the 32nd-nearest gas neighbour), FP32-mixed
form, KDK at the box's Courant step, inputs resident in HBM (about 20 GB of
state, far larger than L2).  Beside it on the same box: the plain FP64 form,
the end-to-end rate through the C ABI with host buffers, the oracle on a
sample, and the 2 x 128^3 Gaussian-field box as a secondary field.

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
# 2, add/mul = 1, sqrt/rsqrt/exp/reciprocal = 1).  Units: density and moments
# per ordered gather pair (self included: each target sums its own set, by
# definition); hydro and gravity per UNORDERED pair (the method's force is
# one evaluation per pair, F_ji = -F_ij; the gather kernels form it from both
# sides, and that second evaluation is not counted as work).  Pairs outside
# the support (leaf-pair overlap) are not counted either.
FLOP_PER_PAIR = {"density": 22, "moments": 125, "hydro": 183, "gravity": 41}

# DRAM bytes (read + write) per particle of one launch of the gravity pass,
# from an ncu capture of gravity_sym_k (each pair once) on the clustered generator at 2 x 64^3
# with 8 dense cores (32,768 particles per core, as in the 2 x 256^3 box),
# leaf capacity 128, scaled to the launch by the particles it processes.  They
# describe the kernels of the csrc/passes.cu with this SHA-256 only; for any
# other source the bench reports no traffic.
TRAFFIC_SOURCE_SHA256 = "33fb3598363ca272e92f6cca363c41703564eb8ef8ff1fe9763c9c4ccce7df80"
TRAFFIC_BYTES_PER_PARTICLE = {"gravity_pairs_once": 79.7}


# the crk_create flag that switches each pass to its pairs-once form (0: none)
_ONCE_FLAG = {"tree": 0, "pairs": 0, "density": 0, "moments": 0, "hydro": 8, "gravity": 2, "kdk": 0}


def _form_flags(crk, form: int) -> int:
    """crk_create flags of an autotuner decomposition (a bit set)."""
    return ((crk.CRK_FLAG_GRAVITY_PAIRS_ONCE if form & crk.CRK_GRAVITY_PAIRS_ONCE else 0) |
            (crk.CRK_FLAG_HYDRO_PAIRS_ONCE if form & crk.CRK_HYDRO_PAIRS_ONCE else 0))


def _form_names(crk, form: int) -> dict:
    return {"gravity_form": "pairs_once" if form & crk.CRK_GRAVITY_PAIRS_ONCE else "gather",
            "hydro_form": "pairs_once" if form & crk.CRK_HYDRO_PAIRS_ONCE else "gather"}


def _tune_summary(crk, cap: int, form: int, grid: dict, digits: int) -> dict:
    """The autotuner's choice and its grid, keys 'capacity/gravity form/hydro form'."""
    short = lambda f: "/".join(v for v in _form_names(crk, f).values())
    return dict({"leaf_cap": cap, "flags": _form_flags(crk, form)}, **_form_names(crk, form),
                force_evaluation_ms={f"{c}/{short(f)}": round(v, digits) for (c, f), v in grid.items()})


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


def fp32_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    """SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock (GB300: 152 SMs)."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def algorithmic_pairs(counts, gas, list_entries=None):
    """Pair counts of one force evaluation in the units of FLOP_PER_PAIR:
    density and moments over ordered gather pairs with self, hydro over
    unordered union pairs (r < max(2h_i, 2h_j); from the list entries of the
    counted evaluation, which hold every target's union set and itself, else
    from the gather sets, which equal the union sets when h is uniform),
    gravity over unordered pairs within r_cut."""
    n_gas = int(gas.sum())
    gather = int(counts["nbr_count"][gas].sum())
    union_ordered = (int(list_entries) - n_gas) if list_entries else gather
    return {"density": gather + n_gas, "moments": gather + n_gas, "hydro": union_ordered // 2,
            "gravity": int(counts["grav_count"].sum()) // 2}


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


def oracle_sample(box, size: int, seed: int = 7):
    """The CPU oracle as it stands on a bounded sample of a box: the forces of
    `size` seeded random particles (both species in proportion), with every
    quantity they depend on (the densities, moments and corrections of their
    neighbours and of those neighbours' neighbours) evaluated too, over the
    whole box's particles.  Returns the timing and the sampled outputs."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(box.n, size=min(size, box.n), replace=False))
    op = oracle.make_params(**box.params())
    t0 = time.perf_counter()
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, sample=idx)
    secs = time.perf_counter() - t0
    return idx, ref, secs


def cpu_baseline(box, size: int, label: str):
    """particles/s of the oracle on a sample of the box (sampled particles
    over the time of their force evaluation, which is the bulk of a step);
    also returns the oracle's sampled outputs for the parity check."""
    import oracle

    idx, ref, secs = oracle_sample(box, size)
    return ({"value": len(idx) / secs, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
             "sample": f"forces of {len(idx)} seeded random particles of the {label} box with everything "
                       f"they depend on (neighbour densities, moments, corrections), {secs:.1f} s"},
            idx, ref)


def serve_bench(crk, wl, args):
    """The serving workload: the first `count` requests of the 2,000-request
    stream (n log-uniform in [16, 128], 20 KDK steps at dt = 1e-3, FP32-mixed,
    150 GB budget, size classes of the service).  A closed-loop calibration
    batch fixes the saturated throughput; Poisson arrivals are then issued at
    70% of it and the service reports each request's submit-to-completion
    latency.  Request boxes are generated on host threads ahead of their
    arrival (the stream holds ~1.3 G particles in all, too many to generate
    up front).  Submission stops once --serve-seconds have passed; the line
    says how many requests ran.  Beside it, sequential plain-FP64 solves (one
    handle per request, one box per launch, the same 20 KDK steps) of a few of
    the requests give the FP64 rate."""
    import concurrent.futures as cf
    import resource

    count = args.serve_requests
    reqs = wl.serving_requests(2000)[:count]
    steps = 20
    svc = crk.crk_service_create(150 * 10**9, max_slots=64, precision=crk.CRK_MIXED,
                                 leaf_cap=args.serve_leaf_cap, lane_priority=args.serve_priority)
    gen = lambda r: wl.gaussian_field_box(r[0], seed=r[1])
    ex = cf.ThreadPoolExecutor(12)

    def submit(b):
        return crk.crk_submit(svc, crk.box_physics(b), b.pos, b.vel, b.mass, b.u, b.h, b.species,
                              b.dt, steps)

    try:
        # calibration: a closed batch of the first requests, all submitted at once
        ncal = min(32, count)
        calib = list(ex.map(gen, reqs[:ncal]))
        t0 = time.perf_counter()
        tk = [submit(b) for b in calib]
        for t, b in zip(tk, calib):
            crk.crk_poll(svc, t, b.n, -1)
        t_cal = time.perf_counter() - t0
        capacity = ncal / t_cal                       # requests/s when saturated
        rate = 0.7 * capacity
        arrivals = wl.poisson_arrivals(count, rate, seed=5)
        # boxes generated in order, at most `ahead` requests before their
        # arrival, and dropped once submitted (the stream does not fit in
        # host memory at once)
        ahead = 48
        futs = {k: ex.submit(gen, reqs[k]) for k in range(min(ahead, count))}
        tickets, sizes, late = [], [], 0
        res = {}          # latencies of finished requests, collected as they finish
        outstanding = []

        def collect(wait: bool):
            keep = []
            for k in outstanding:
                r = crk.crk_poll(svc, tickets[k], sizes[k], -1 if wait else 0, state=False)
                if r is None:
                    keep.append(k)
                else:
                    res[k] = r
            outstanding[:] = keep

        t0 = time.perf_counter()
        for k, a in enumerate(arrivals):
            if time.perf_counter() - t0 > args.serve_seconds:
                break
            while time.perf_counter() - t0 < a:
                time.sleep(min(1e-3, max(0.0, a - (time.perf_counter() - t0))))
            b = futs.pop(k).result()
            if k + ahead < count:
                futs[k + ahead] = ex.submit(gen, reqs[k + ahead])
            late += (time.perf_counter() - t0) > a + 0.05
            tickets.append(submit(b))
            sizes.append(b.n)
            outstanding.append(k)
            del b
            collect(False)
        for f in futs.values():
            f.cancel()
        futs.clear()
        collect(True)
        res = [res[k] for k in range(len(tickets))]
        wall = time.perf_counter() - t0
    finally:
        crk.crk_service_destroy(svc)
        ex.shutdown(wait=True, cancel_futures=True)
    lat = np.array([r["latency_ns"] for r in res]) / 1e6
    que = np.array([r["queue_ns"] for r in res]) / 1e6
    psteps = sum(sizes) * steps

    # sequential plain FP64, one request at a time, the same 20 KDK steps
    seq = [gen(r) for r in reqs[:min(args.serve_fp64, count)]]
    t64 = 0.0
    p64 = 0
    for b in seq:
        s = crk.Sim(crk.box_physics(b), leaf_cap=64, precision=crk.CRK_FP64)
        s.load(b)
        t1 = time.perf_counter()
        s.step(b.dt, steps)
        s.state()
        t64 += time.perf_counter() - t1
        p64 += b.n * steps
        s.close()
    small = np.array(sizes) < 65536
    bounds = [0, 65536, 524288, 1 << 62]
    per_class = []
    for k in range(3):
        sel = (np.array(sizes) >= bounds[k]) & (np.array(sizes) < bounds[k + 1])
        if sel.any():
            per_class.append({"particles": f"[{bounds[k]}, {bounds[k + 1] if k < 2 else 'inf'})",
                              "requests": int(sel.sum()),
                              "p50_ms": round(float(np.percentile(lat[sel], 50)), 3),
                              "p99_ms": round(float(np.percentile(lat[sel], 99)), 3)})
    return {"requests": len(res), "of": 2000, "steps_per_request": steps,
            "per_size_class": per_class,
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "p99_over_p50": round(float(np.percentile(lat, 99) / np.percentile(lat, 50)), 3),
            "p50_ms_small_jobs": round(float(np.percentile(lat[small], 50)), 3) if small.any() else None,
            "queue_p50_ms": round(float(np.percentile(que, 50)), 3),
            "value": psteps / wall, "unit": UNIT, "wall_s": round(wall, 2),
            "arrival_rate_per_s": round(rate, 3), "load": 0.7, "late_submissions": int(late),
            "host_peak_rss_gb": round(resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 2**20, 1),
            "calibration": {"requests": ncal, "seconds": round(t_cal, 3)},
            "size_classes": "3 (below 65,536 particles; below 524,288; the rest)",
            "lane_priority": args.serve_priority,
            "fp64_sequential": {"value": p64 / t64 if t64 else None, "unit": UNIT, "requests": len(seq),
                                "steps_per_request": steps}}


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


def fp64_pass_rates(tim, pairs, peak_tflops: float, peak_source: str):
    """Per-phase times of the timed FP64 evaluations and each pair pass's
    algorithmic rate, also as a share of the measured FP64 FMA rate."""
    calls = max(tim["calls"], 1)
    rates = {k: pairs[k] * FLOP_PER_PAIR[k] / (tim[k + "_ms"] / calls / 1e3) / 1e12
             for k in ("density", "moments", "hydro", "gravity") if tim[k + "_ms"] > 0}
    return {"breakdown_ms": {k: round(tim[k] / calls, 3) for k in
                             ("tree_ms", "pairs_ms", "density_ms", "moments_ms", "hydro_ms",
                              "gravity_ms", "kdk_ms")},
            "pass_tflops": {k: round(v, 4) for k, v in rates.items()},
            "pass_of_fp64_peak": {k: round(v / peak_tflops, 4) for k, v in rates.items()},
            "fp64_peak": {"value": round(peak_tflops, 4), "unit": "TFLOP/s", "source": peak_source}}


def pair_census(tim, gather_pairs: int, grav_ordered: int, n: int):
    """Evaluated / algorithmic pairs of the counted evaluation: candidate
    tests in lane slots (a warp tests its up to 32 targets against every staged
    candidate) per in-range ordered pair, the hydro list entries per gather
    pair (self included), and the share of walked list slots that hold an
    entry."""
    grav = grav_ordered + n                   # each target is also tested against itself
    r = lambda a, b: round(a / b, 3) if b else None
    return {"gravity": {"tested_slots": tim["tests_grav"], "target_slots": tim["tests_grav_target"],
                        "in_range": grav, "tested_per_in_range": r(tim["tests_grav"], grav),
                        "target_slots_per_in_range": r(tim["tests_grav_target"], grav)},
            "hydro_fill": {"tested_slots": tim["tests_hydro"], "list_entries": tim["list_entries"],
                           "gather_pairs": gather_pairs,
                           "tested_per_entry": r(tim["tests_hydro"], tim["list_entries"]),
                           "entries_per_gather_pair": r(tim["list_entries"], gather_pairs)},
            "list_walk": {"slots": tim["list_slots"], "entries": tim["list_entries"],
                          "entry_share": r(tim["list_entries"], tim["list_slots"])},
            "note": "lane slots of one counted force evaluation; in-range gravity pairs are ordered and "
                    "include each target's self test"}


def run_precision(args):
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
            runs[name]["census"] = pair_census(crk.crk_get_timings(s.handle),
                                               int(cnt["nbr_count"][gas].sum()) + int(gas.sum()),
                                               int(cnt["grav_count"].sum()), box.n)
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


def batched_leg(crk, wl, steps: int, warmup: int, stream) -> dict:
    """The batched workload: 64 independent periodic boxes of 2 n^3 particles,
    n drawn (seed 2) from {16, 24, 32, 48, 64}, box b from the Gaussian-field
    generator with seed 1000 + b, all in one handle (one tree and one launch
    per pass for every box), FP32-mixed, leaf capacity and gravity form chosen
    by the library's autotuner; the timed steps replayed from a CUDA graph
    (persistent pass launches draining one device work queue of every box's
    target groups).  Beside it the plain FP64 form one box per handle, run
    one box after another, on the first 8 boxes."""
    import torch

    boxes = wl.batched_boxes(64, seed=2)
    cat = wl.concat_boxes(boxes)
    N = int(cat["offsets"][-1])
    phys = [crk.box_physics(b) for b in boxes]
    dts = [b.dt for b in boxes]
    sim = crk.Sim(phys[0], leaf_cap=128, precision=crk.CRK_MIXED, stream=stream)
    crk.crk_load_boxes(sim.handle, [b.n for b in boxes], phys, cat["pos"], cat["vel"], cat["mass"],
                       cat["u"], cat["h"], cat["species"])
    sim.n = N
    best, form, grid = crk.crk_autotune_ex(sim.handle, (32, 64, 128))
    crk.crk_step_boxes(sim.handle, dts, warmup)
    crk.crk_set_timing(sim.handle, False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    crk.crk_step_boxes(sim.handle, dts, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    tg = crk.crk_get_timings(sim.handle)
    crk.crk_set_timing(sim.handle, True)        # per-phase times from host-sized steps
    crk.crk_step_boxes(sim.handle, dts, 2)
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
    return {"workload": "batched: 64 Gaussian-field boxes 2 n^3, n in {16,24,32,48,64} (seed 2), one handle, "
                        "FP32-mixed, KDK dt=1e-3",
            "particles": N, "boxes": len(boxes), "value": N / (ms / 1e3), "unit": UNIT,
            "ms_per_step": round(ms, 3), "steps": steps,
            "graph": {"steps": int(tg["steps"]), "graph_steps": int(tg["graph_steps"]),
                      "host_syncs": int(tg["host_syncs"]), "overflows": int(tg["graph_overflows"])},
            "autotune": _tune_summary(crk, best, form, grid, 3),
            "breakdown_ms": {k: round(tim[k] / calls, 4) for k in
                             ("tree_ms", "pairs_ms", "density_ms", "moments_ms", "hydro_ms", "gravity_ms",
                              "kdk_ms")},
            "gpu_launches_per_host_sized_step": int(tim["launches"]) // max(int(tim["calls"]), 1),
            "fp64_one_box_per_launch": {"value": p64 / t64, "unit": UNIT, "boxes": 8, "steps": 1}}


def run_batched(args):
    """The batched workload as its own line (see batched_leg)."""
    import torch

    from paper_2510_03557_gb300 import crk
    from paper_2510_03557_gb300 import workloads as wl

    torch.cuda.set_device(0)
    crk.lib()
    stream = torch.cuda.Stream()
    with ClockSampler(0) as clocks:
        b = batched_leg(crk, wl, args.steps, args.warmup, stream)
    line = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "particles": b["particles"], "boxes": b["boxes"],
                       "leaf_cap": b["autotune"]["leaf_cap"]},
            "batched": b, "clocks": clocks.summary()}
    print(json.dumps(line))


def headline_config(args, world: int) -> dict:
    """The headline workload's config, as both arms report it: the clustered
    2 x n^3 box of the generator (seed 3), KDK at the box's Courant step."""
    n = 2 * args.n ** 3
    return {"workload": f"clustered 2x{args.n}^3 (half uniform, half in {getattr(args, 'nsphere', 512)} Plummer "
                        f"spheres of scale 0.002, kNN h), FP32-mixed, KDK steps at the box's Courant dt",
            "particles": n,
            "leaf_cap": "autotuned over (64, 128) with the pair decompositions" if args.autotune else args.leaf_cap,
            "rebuild_every": args.rebuild_every,
            "parallelism": f"replicas{world}",
            "l2": f"inputs larger than L2 (~{n * 600 / 1e9:.1f} GB resident state)"}


def run_reference(args):
    """The reference arm: the oracle as it stands, on the host cores, on a
    bounded sample of the headline workload each step (the forces of
    --cpu-sample seeded random particles of the same box with everything they
    depend on; --ref-sample particles), on the headline's config, metric and
    unit.  Under torchrun
    only rank 0 runs; the other ranks exit without work."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2510_03557_gb300 import workloads as wl

    box = wl.clustered_box(args.n, seed=3, nsphere=args.nsphere)
    label = f"clustered 2x{args.n}^3"
    steps = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline(box, args.ref_sample, label)
    for _ in range(args.steps):
        cb, _, _ = cpu_baseline(box, args.ref_sample, label)
        steps.append(cb["value"])
    value = statistics.median(steps) if steps else 0.0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": headline_config(args, args.gpus),
            "cpu_baseline": dict(cb or {}, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gaussian(crk, wl, args, stream, timed_steps: int):
    """The 2 x 128^3 Gaussian-field box (P(k) ~ k^-2, 0.3-cell rms
    displacement, ~270 gas neighbours), the same mixed KDK steps: a
    secondary field of the headline line (and, with --workload gaussian, a
    line of its own)."""
    import torch

    box = wl.gaussian_field_box(args.gauss_n, seed=1)
    gas = box.species == wl.GAS
    sim = crk.Sim(crk.box_physics(box), leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream,
                  rebuild_every=args.rebuild_every)
    sim.load(box)
    counts = sim.forces(counts=True)
    tim0 = crk.crk_get_timings(sim.handle)
    pairs = algorithmic_pairs(counts, gas, tim0["list_entries"])
    for _ in range(3):
        sim.step(box.dt, 1)
    crk.crk_set_timing(sim.handle, False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(box.dt, timed_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / timed_steps
    graph_steps = int(crk.crk_get_timings(sim.handle)["graph_steps"])
    crk.crk_set_timing(sim.handle, True)       # per-phase times from host-sized steps
    sim.step(box.dt, 3)
    tim = crk.crk_get_timings(sim.handle)
    calls = max(tim["calls"], 1)
    out = {"workload": f"gaussian-field 2x{args.gauss_n}^3, FP32-mixed, KDK dt={box.dt}", "particles": box.n,
           "value": box.n / (ms / 1e3), "unit": UNIT, "ms_per_step": round(ms, 4), "steps": timed_steps,
           "graph_steps": graph_steps,
           "breakdown_ms": {k: round(tim[k] / calls, 4) for k in
                            ("tree_ms", "pairs_ms", "density_ms", "moments_ms", "hydro_ms", "gravity_ms",
                             "kdk_ms")},
           "pass_tflops": {k: round(pairs[k] * FLOP_PER_PAIR[k] / (tim[k + "_ms"] / calls / 1e3) / 1e12, 3)
                           for k in ("density", "moments", "hydro", "gravity")},
           "pairs_per_step": pairs,
           "pair_census": pair_census(tim0, pairs["density"], int(counts["grav_count"].sum()), box.n),
           "leaves": int(tim["nleaves"])}
    fof = None
    if not args.no_extras:
        torch.cuda.synchronize()
        t_f = time.perf_counter()
        _, n_groups = crk.crk_fof(sim.handle, 0.2 / args.gauss_n, 1, box.n)
        fof = {"ms": round((time.perf_counter() - t_f) * 1e3, 3), "groups": n_groups,
               "linking_length": 0.2 / args.gauss_n, "species": "dm",
               "note": "host wall time of crk_fof: tree build, links, labels, copy-out"}
    sim.close()
    mesh = None
    if not args.no_extras:
        # the same KDK step with the long-range mesh (FP64 PM, n^3 cells)
        smesh = crk.Sim(crk.box_physics(box), leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream,
                        rebuild_every=args.rebuild_every, pm_grid=args.gauss_n)
        smesh.load(box)
        smesh.step(box.dt, 2)
        crk.crk_set_timing(smesh.handle, True)
        smesh.step(box.dt, 3)
        tmesh = crk.crk_get_timings(smesh.handle)
        mcalls = max(tmesh["calls"], 1)
        mesh = {"pm_grid": args.gauss_n, "pm_ms": round(tmesh["pm_ms"] / mcalls, 4),
                "step_ms": round(tmesh["total_ms"] / mcalls, 4),
                "note": "per KDK step, CUDA events on the handle's stream: deposit, cuFFT forward, "
                        "Green's function, 3 cuFFT inverse, gather (FP64)"}
        smesh.close()
    out["fof"] = fof
    out["long_range_mesh"] = mesh
    return out


def parity_on_sample(out, ref, idx, gas):
    """Relative L2 and the worst particle's relative error of a GPU form's
    outputs against the oracle on the sampled particles."""
    gi = idx[gas[idx]]
    res = {}
    for k, ok, sel in (("acc", "acc", idx), ("dudt", "dudt", gi), ("rho", "rho", gi), ("A", "A", gi),
                       ("B", "B", gi), ("gradA", "dA", gi), ("gradB", "dB", gi)):
        a = np.asarray(out[k][sel], np.float64).reshape(len(sel), -1)
        b = np.asarray(ref[ok][sel], np.float64).reshape(len(sel), -1)
        nb = np.linalg.norm(b, axis=1)
        floor = 1e-6 * float(np.sqrt(np.mean(nb * nb))) if len(nb) else 0.0
        per = np.linalg.norm(a - b, axis=1) / np.maximum(nb + floor, 1e-300)
        res[k] = {"rel_l2": _rel_l2(a, b), "worst_particle": float(per.max()) if len(per) else 0.0}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "gaussian", "precision", "batched", "bins"],
                    help="headline: the clustered 2 x n^3 line; gaussian: the 2 x 128^3 box alone; "
                         "precision: FP64 and mixed KDK on the clustered box with per-output errors; "
                         "batched: 64 boxes in one handle; bins: hierarchical steps (each prints its own line)")
    ap.add_argument("--bin-depth", type=int, default=5, help="bins workload: substeps 2^depth")
    ap.add_argument("--bin-eta", type=float, default=0.025)
    ap.add_argument("--bin-courant", type=float, default=0.25)
    ap.add_argument("--sample", type=int, default=64, help="oracle sample of the precision study")
    ap.add_argument("--n", type=int, default=256, help="clustered box: lattice size per species (2 n^3)")
    ap.add_argument("--nsphere", type=int, default=512,
                    help="clustered box: Plummer spheres (8 at n = 64 gives the 32,768-particle cores of "
                         "n = 256 with 512; the small case of the profiles)")
    ap.add_argument("--pairs-once", action="store_true",
                    help="with --no-autotune: gravity with each pair evaluated once")
    ap.add_argument("--hydro-once", action="store_true",
                    help="with --no-autotune: hydro with each union pair evaluated once")
    ap.add_argument("--gauss-n", type=int, default=128, help="Gaussian-field box: 2 n^3 particles")
    ap.add_argument("--leaf-cap", type=int, default=128)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="headline: keep --leaf-cap and the gather gravity instead of the library's autotuner")
    ap.add_argument("--rebuild-every", type=int, default=1,
                    help="sort into new leaves every this many steps (boxes grow in between)")
    ap.add_argument("--fp64-evals", type=int, default=1,
                    help="timed FP64 force evaluations on the headline box (0: skip the FP64 form)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="precision workload: KDK steps of the FP64 form (-1 = as many as the mixed form)")
    ap.add_argument("--cpu-sample", type=int, default=256,
                    help="particles of the oracle's sample in cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=32,
                    help="particles of the oracle's sample in each step of the reference arm")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-gaussian", action="store_true", help="skip the 2 x 128^3 secondary field")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-box batched field")
    ap.add_argument("--no-extras", action="store_true", help="skip the FOF and long-range mesh legs")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream to run (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=700.0,
                    help="stop submitting serving requests after this many seconds")
    ap.add_argument("--serve-fp64", type=int, default=4, help="requests solved one by one in plain FP64")
    ap.add_argument("--serve-leaf-cap", type=int, default=64)
    ap.add_argument("--serve-priority", type=int, default=1, choices=[-1, 0, 1],
                    help="service lane_priority: 1 larger size classes first")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "precision":
        run_precision(args)
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
    stream = torch.cuda.Stream()
    if args.workload == "gaussian":
        g = run_gaussian(crk, wl, args, stream, args.steps)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": g["value"], "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "ms_per_step": g["ms_per_step"], "higher_is_better": True,
                              "dtype": "f32", "data": "synthetic", "config": {"workload": g["workload"]},
                              "gaussian": g}))
        return

    legs = {}
    t_leg = time.perf_counter()

    def leg(name):
        nonlocal t_leg
        now = time.perf_counter()
        legs[name] = round(now - t_leg, 1)
        t_leg = now

    box = wl.clustered_box(args.n, seed=3, nsphere=args.nsphere)
    leg("setup")
    t_gen = legs["setup"]
    N = box.n
    dt = box.dt
    phys = crk.box_physics(box)
    gas = box.species == wl.GAS
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # ---------------- mixed form, device-resident (the headline value)
    head_flags = 0 if args.autotune else ((crk.CRK_FLAG_GRAVITY_PAIRS_ONCE if args.pairs_once else 0) |
                                          (crk.CRK_FLAG_HYDRO_PAIRS_ONCE if args.hydro_once else 0))
    sim = crk.Sim(phys, leaf_cap=args.leaf_cap, precision=crk.CRK_MIXED, stream=stream,
                  rebuild_every=args.rebuild_every, flags=head_flags)
    sim.load(box)
    tune = None
    cap = args.leaf_cap
    if args.autotune:
        # the library's autotuner: leaf capacity x the gravity and hydro pair
        # decompositions
        cap, form, grid = crk.crk_autotune_ex(sim.handle, (64, 128))
        tune = _tune_summary(crk, cap, form, grid, 2)
        head_flags = tune["flags"]
    counts = sim.forces(counts=True)      # untimed: the true pair counts for the roofline
    tim0 = crk.crk_get_timings(sim.handle)
    pairs = algorithmic_pairs(counts, gas, tim0["list_entries"])
    census = pair_census(tim0, pairs["density"], int(counts["grav_count"].sum()), N)
    for _ in range(args.warmup):
        sim.step(dt, 1)
    crk.crk_set_timing(sim.handle, False)     # counters reset; steps replayed from CUDA graphs
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
    tg = crk.crk_get_timings(sim.handle)
    graph = {"steps": int(tg["steps"]), "graph_steps": int(tg["graph_steps"]),
             "host_syncs": int(tg["host_syncs"]), "overflows": int(tg["graph_overflows"]),
             "note": "the timed crk_step call: its first step host-sized, the rest replayed from a CUDA graph of "
                     "two steps (persistent pass launches over device work queues); host synchronisations of "
                     "the whole call"}
    # per-phase times (CUDA events between the phases need host-sized steps)
    crk.crk_set_timing(sim.handle, True)
    sim.step(dt, max(2, min(args.steps, 3)))
    tim = crk.crk_get_timings(sim.handle)
    per_pass_ms = {"density": tim["density_ms"], "moments": tim["moments_ms"],
                   "hydro": tim["hydro_ms"], "gravity": tim["gravity_ms"]}
    calls = max(tim["calls"], 1)
    dom = max(per_pass_ms, key=per_pass_ms.get)
    dom_ms = per_pass_ms[dom] / calls
    clk = clocks.summary()
    peaks, peak_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_max, sms)
    fma32 = crk.crk_fma_peak(crk.CRK_MIXED, stream)
    fma64 = crk.crk_fma_peak(crk.CRK_FP64, stream)
    achieved = pairs[dom] * FLOP_PER_PAIR[dom] / (dom_ms / 1e3) / 1e12
    pass_tflops = {k: pairs[k] * FLOP_PER_PAIR[k] / (per_pass_ms[k] / calls / 1e3) / 1e12
                   for k in per_pass_ms}
    breakdown = {k: round(v / calls, 4) for k, v in
                 (("tree_ms", tim["tree_ms"]), ("pairs_ms", tim["pairs_ms"]),
                  ("density_ms", tim["density_ms"]), ("moments_ms", tim["moments_ms"]),
                  ("hydro_ms", tim["hydro_ms"]), ("gravity_ms", tim["gravity_ms"]),
                  ("kdk_ms", tim["kdk_ms"]))}
    launches = int(tim["launches"])
    fof = None
    if not args.no_extras:
        # friends-of-friends halos of the dark matter at b = 0.2 mean spacings
        # on the clustered state after the steps (a new tree, then links)
        torch.cuda.synchronize()
        t_f = time.perf_counter()
        grp, n_groups = crk.crk_fof(sim.handle, 0.2 / args.n, 1, N)
        _, sizes = np.unique(grp[grp >= 0], return_counts=True)
        fof = {"ms": round((time.perf_counter() - t_f) * 1e3, 3), "groups": n_groups,
               "groups_20_or_more": int(np.sum(sizes >= 20)), "largest": int(sizes.max()) if len(sizes) else 0,
               "linking_length": 0.2 / args.n, "species": "dm",
               "note": "host wall time of crk_fof: tree build, links, labels, copy-out"}
    sim.close()
    leg("mixed")

    # ---------------- FP64 plain form on the same box, the same state
    fp64 = None
    out64 = None
    if args.fp64_evals > 0:
        s64 = crk.Sim(phys, leaf_cap=cap, precision=crk.CRK_FP64, stream=stream)
        s64.load(box)
        crk.crk_set_timing(s64.handle, True)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_evals):
            out64 = s64.forces(counts=False)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = max_over_ranks(f0.elapsed_time(f1)) / args.fp64_evals   # includes the copy-out
        tim64 = crk.crk_get_timings(s64.handle)
        dev64 = tim64["total_ms"] / max(tim64["calls"], 1)
        fp64 = {"value": world * N / (dev64 / 1e3), "unit": UNIT, "ms_per_force_evaluation": round(dev64, 2),
                "wall_ms_with_copy_out": round(t64, 2), "evaluations": args.fp64_evals, "dtype": "f64",
                "rate_from": "device time of a force evaluation (tree, lists, D, M, C, H, G); a KDK step adds "
                             "only its FP64 kicks and drift (kdk_ms of the mixed form)",
                "mixed_over_fp64": round(value / (world * N / (dev64 / 1e3)), 2)}
        fp64.update(fp64_pass_rates(tim64, pairs, fma64, "crk_fma_peak: FP64 FMA chains on this device"))
        s64.close()
        leg("fp64")
    precision = None
    if out64 is not None:
        # the mixed form against the FP64 form at the loaded state (both forms'
        # first force evaluation), relative L2 per output over every particle
        precision = {k: _rel_l2(counts[k][sel], out64[k][sel]) for k, sel in
                     (("acc", slice(None)), ("dudt", gas), ("rho", gas), ("A", gas), ("B", gas),
                      ("gradA", gas), ("gradB", gas))}
        del out64

    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        se = crk.Sim(phys, leaf_cap=cap, precision=crk.CRK_MIXED, stream=stream,
                     flags=head_flags)
        se.load(box)
        se.step(dt, 1)
        pin = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
        hp, hv, hu = pin((N, 3)), pin((N, 3)), pin(N)
        crk.crk_get_state(se.handle, hp, hv, hu)
        k_e2e = max(2, min(args.steps, 3))
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
        del hp, hv, hu
        leg("e2e")

    gaussian = None
    if not args.no_gaussian:
        gaussian = run_gaussian(crk, wl, args, stream, max(2, min(args.steps, 10)))
        leg("gaussian")

    batched = None
    if not args.no_batched:
        batched = batched_leg(crk, wl, max(3, min(args.steps, 10)), 2, stream)
        leg("batched")

    serving = None
    if args.serve_requests > 0:
        serving = serve_bench(crk, wl, args)
        leg("serving")

    cb = None
    sample_parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb, idx, ref = cpu_baseline(box, args.cpu_sample, f"clustered 2x{args.n}^3")
        sample_parity = {"particles": int(len(idx)), "mixed": parity_on_sample(counts, ref, idx, gas),
                         "oracle_rc": int(ref["rc"])}
        leg("cpu_baseline")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": headline_config(args, world),
            "roofline": {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3),
                         "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                         "traffic": _traffic(dom + ("_pairs_once" if head_flags & _ONCE_FLAG[dom]
                                                    else "_gather"), N, cap),
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on "
                                           "the clustered generator at 2x64^3 with 8 dense cores, scaled by "
                                           "particles (null when the kernel source or leaf capacity differs from "
                                           "the captured one)",
                         "work": f"{FLOP_PER_PAIR[dom]} flop per "
                                 f"{'unordered' if dom in ('hydro', 'gravity') else 'ordered'} in-range pair",
                         "peak_source": f"{sms} SMs (device query) x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                        f"({peak_kind} sm_max_mhz)",
                         "fma_probe_tflops": {"fp32": round(fma32, 3), "fp64": round(fma64, 4)}},
            "pass_tflops": {k: round(v, 3) for k, v in pass_tflops.items()},
            "pass_of_fp32_peak": {k: round(v / peak, 4) for k, v in pass_tflops.items()},
            "pairs_per_step": pairs,
            "pair_census": census,
            "leaves": int(tim["nleaves"]), "leaf_pairs": {"hydro": int(tim["pairs_hydro"]),
                                                          "gravity": int(tim["pairs_grav"])},
            "breakdown_ms": breakdown,
            "breakdown_note": "per-phase CUDA-event times of host-sized steps after the timed region "
                              "(the roofline's kernel time is the same kernel's in the replayed steps)",
            "graph": graph,
            "autotune": tune,
            "dt": dt,
            "setup_s": round(t_gen, 1),
            "fp64_plain": fp64,
            "mixed_vs_fp64_rel_l2": precision,
            "oracle_sample_parity": sample_parity,
            "fof": fof,
            "gaussian_2x128": gaussian,
            "batched_64_boxes": batched,
            "serving": serving,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cb,
            "leg_wall_s": legs,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
