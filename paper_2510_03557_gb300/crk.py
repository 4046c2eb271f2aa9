"""Thin Python binding of libcrk's C ABI (include/crk.h), argument marshalling
only: every step of the solver runs in the library's CUDA kernels.

Arrays may be NumPy arrays (host memory) or CUDA torch tensors (device
memory); one call takes one kind.  There is no CPU fallback: importing the
binding without a built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcrk.so")

CRK_OK = 0
CRK_EINVAL = -1
CRK_ENOMEM = -2
CRK_ECUDA = -3
CRK_EOVERFLOW = -4
CRK_ESINGULAR = -5
CRK_EPENDING = -6
CRK_ETIMEOUT = -7
CRK_ENOTFOUND = -8
CRK_ECANCELED = -9
CRK_FP64 = 0
CRK_MIXED = 1
CRK_WENDLAND_C4 = 0
CRK_MEM_HOST = 0
CRK_MEM_DEVICE = 1
CRK_FLAG_GRAVITY_PAIRS_ONCE = 2
CRK_FLAG_NO_GRAPH = 4
CRK_FLAG_HYDRO_PAIRS_ONCE = 8
CRK_GRAVITY_GATHER = 0
CRK_GRAVITY_PAIRS_ONCE = 1
CRK_HYDRO_PAIRS_ONCE = 2
CRK_DM = 0
CRK_GAS = 1

# Every function of the C ABI.
ABI = ("crk_create", "crk_load", "crk_load_boxes", "crk_forces", "crk_step", "crk_step_boxes",
       "crk_get_state", "crk_set_state", "crk_get_sums", "crk_get_size", "crk_set_timing", "crk_get_timings",
       "crk_destroy", "crk_fof", "crk_pm_accel", "crk_step_bins", "crk_get_bins",
       "crk_autotune", "crk_autotune_ex", "crk_service_create", "crk_submit", "crk_poll", "crk_service_destroy",
       "crk_service_snapshot", "crk_service_cancel",
       "crk_neighbours_noalloc", "crk_get_tree", "crk_fma_peak", "crk_last_error")
CRK_NOALLOC_MAX_N = 262144


class CrkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libcrk error {code}: {msg}")
        self.code = code


class Physics(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("box", "G", "gamma", "r_cut", "r_split",
                                                "eps_soft", "av_alpha", "av_beta", "av_eps2",
                                                "u_floor")]


class Params(ctypes.Structure):
    _fields_ = [("phys", Physics), ("kernel", ctypes.c_int), ("leaf_cap", ctypes.c_int),
                ("precision", ctypes.c_int), ("cm_level", ctypes.c_int), ("flags", ctypes.c_int),
                ("rebuild_every", ctypes.c_int), ("pm_grid", ctypes.c_int), ("graph_margin_pct", ctypes.c_int)]


class Outputs(ctypes.Structure):
    _fields_ = [("acc", ctypes.c_void_p), ("dudt", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("gradA", ctypes.c_void_p),
                ("gradB", ctypes.c_void_p), ("nbr_count", ctypes.c_void_p),
                ("nbr_hash", ctypes.c_void_p), ("grav_count", ctypes.c_void_p),
                ("grav_hash", ctypes.c_void_p), ("mem", ctypes.c_int), ("reserved", ctypes.c_int),
                ("momentum_rate", ctypes.c_double * 3), ("energy_rate", ctypes.c_double)]


class Timings(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("tree_ms", "pairs_ms", "density_ms", "moments_ms",
                                                "hydro_ms", "gravity_ms", "kdk_ms", "total_ms")] + \
               [(k, ctypes.c_int64) for k in ("calls", "pairs_hydro", "pairs_grav", "nleaves",
                                               "launches")] + [("pm_ms", ctypes.c_double)] + \
               [(k, ctypes.c_int64) for k in ("tests_hydro", "list_entries", "tests_grav",
                                               "tests_grav_target", "list_slots", "steps", "graph_steps",
                                               "host_syncs", "graph_overflows")]


class Tree(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("n", "nleaf", "npair_hydro", "npair_grav")] + \
               [(k, ctypes.c_void_p) for k in ("order", "leaf_start", "leaf_count", "leaf_species",
                                                "leaf_centre", "leaf_half", "hydro_row", "hydro_col",
                                                "grav_row", "grav_col")]


class ServiceParams(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("precision", ctypes.c_int), ("leaf_cap", ctypes.c_int), ("device", ctypes.c_int),
                ("snapshot_every", ctypes.c_int), ("size_classes", ctypes.c_int),
                ("lane_priority", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


class Job(ctypes.Structure):
    _fields_ = [("phys", Physics), ("n", ctypes.c_int64), ("pos", ctypes.c_void_p),
                ("vel", ctypes.c_void_p), ("mass", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("species", ctypes.c_void_p), ("dt", ctypes.c_double),
                ("nsteps", ctypes.c_int), ("steps_done", ctypes.c_int), ("acc", ctypes.c_void_p),
                ("dudt", ctypes.c_void_p)]


class JobSnapshot(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("acc", ctypes.c_void_p), ("dudt", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("steps_done", ctypes.c_int), ("reserved", ctypes.c_int)]


class JobResult(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("latency_ns", ctypes.c_int64), ("queue_ns", ctypes.c_int64),
                ("status", ctypes.c_int), ("reserved", ctypes.c_int)]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libcrk.so (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcrk.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name in ABI:
            getattr(L, name).restype = ctypes.c_int
        L.crk_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int) -> int:
    if rc != CRK_OK:
        raise CrkError(rc, lib().crk_last_error().decode())
    return rc


def physics(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.1, r_split=0.02, eps_soft=0.0,
            av_alpha=1.0, av_beta=2.0, av_eps2=0.01, u_floor=1e-10, **_ignored) -> Physics:
    return Physics(box, G, gamma, r_cut, r_split, eps_soft, av_alpha, av_beta, av_eps2, u_floor)


def params(phys: Physics | None = None, leaf_cap=64, precision=CRK_MIXED, cm_level=0,
           kernel=CRK_WENDLAND_C4, rebuild_every=1, pm_grid=0, flags=0, graph_margin_pct=0) -> Params:
    p = Params()
    p.graph_margin_pct = graph_margin_pct
    p.phys = phys if phys is not None else physics()
    p.kernel = kernel
    p.flags = flags
    p.leaf_cap = leaf_cap
    p.precision = precision
    p.cm_level = cm_level
    p.rebuild_every = rebuild_every
    p.pm_grid = pm_grid
    return p


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, mem, keepalive) of a NumPy array or CUDA tensor."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch

        tdt = {np.float64: torch.float64, np.uint8: torch.uint8, np.int32: torch.int32,
               np.uint64: torch.uint64 if hasattr(torch, "uint64") else torch.int64}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {tdt}")
        if not a.is_cuda:
            a = a.numpy()
        else:
            return ctypes.c_void_p(a.data_ptr()), CRK_MEM_DEVICE, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), CRK_MEM_HOST, arr


def _mem_of(*ms):
    ms = {m for m in ms if m is not None}
    if len(ms) > 1:
        raise TypeError("mix of host and device arrays in one call")
    return ms.pop() if ms else CRK_MEM_HOST


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))


# ----------------------------------------------------------------- calls
def crk_create(prm: Params, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().crk_create(ctypes.byref(prm), _stream_handle(stream), ctypes.byref(h)))
    return h


def crk_load(sim, pos, vel, mass, u, h, species):
    args = [_ptr(pos, np.float64), _ptr(vel, np.float64), _ptr(mass, np.float64),
            _ptr(u, np.float64), _ptr(h, np.float64), _ptr(species, np.uint8)]
    mem = _mem_of(*[a[1] for a in args])
    n = int(np.prod(pos.shape) // 3) if pos is not None else 0
    _check(lib().crk_load(sim, ctypes.c_int64(n), *[a[0] for a in args], ctypes.c_int(mem)))


def crk_load_boxes(sim, counts, phys_list, pos, vel, mass, u, h, species):
    nbox = len(counts)
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    ph = (Physics * nbox)(*phys_list)
    args = [_ptr(pos, np.float64), _ptr(vel, np.float64), _ptr(mass, np.float64),
            _ptr(u, np.float64), _ptr(h, np.float64), _ptr(species, np.uint8)]
    mem = _mem_of(*[a[1] for a in args])
    _check(lib().crk_load_boxes(sim, ctypes.c_int(nbox), cnt.ctypes.data_as(ctypes.c_void_p), ph,
                                *[a[0] for a in args], ctypes.c_int(mem)))


OUTPUT_FIELDS = {"acc": (3, np.float64), "dudt": (1, np.float64), "rho": (1, np.float64),
                 "A": (1, np.float64), "B": (3, np.float64), "gradA": (3, np.float64),
                 "gradB": (9, np.float64), "nbr_count": (1, np.int32), "nbr_hash": (1, np.uint64),
                 "grav_count": (1, np.int32), "grav_hash": (1, np.uint64)}


def crk_forces(sim, **outs):
    """outs: name -> preallocated array (NumPy or CUDA tensor) for any of
    OUTPUT_FIELDS.  Returns (momentum_rate[3], energy_rate)."""
    o = Outputs()
    keep = []
    mems = []
    for name, arr in outs.items():
        if name not in OUTPUT_FIELDS:
            raise KeyError(name)
        if arr is None:
            continue
        p, m, k = _ptr(arr, OUTPUT_FIELDS[name][1])
        if m == CRK_MEM_HOST and k is not arr:
            raise TypeError(f"output {name} must be a contiguous array of {OUTPUT_FIELDS[name][1]}")
        setattr(o, name, p)
        keep.append(k)
        mems.append(m)
    o.mem = _mem_of(*mems)
    _check(lib().crk_forces(sim, ctypes.byref(o)))
    return list(o.momentum_rate), float(o.energy_rate)


def crk_step(sim, dt: float, nsteps: int):
    _check(lib().crk_step(sim, ctypes.c_double(dt), ctypes.c_int(nsteps)))


def crk_step_boxes(sim, dt, nsteps: int):
    d = np.ascontiguousarray(dt, dtype=np.float64)
    _check(lib().crk_step_boxes(sim, d.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(nsteps)))


def crk_get_state(sim, pos=None, vel=None, u=None):
    args = [_ptr(pos, np.float64), _ptr(vel, np.float64), _ptr(u, np.float64)]
    for a, src in zip(args, (pos, vel, u)):
        if a[1] == CRK_MEM_HOST and src is not None and a[2] is not src:
            raise TypeError("state outputs must be contiguous float64 arrays")
    mem = _mem_of(*[a[1] for a in args])
    _check(lib().crk_get_state(sim, *[a[0] for a in args], ctypes.c_int(mem)))


def crk_set_state(sim, pos=None, vel=None, u=None):
    args = [_ptr(pos, np.float64), _ptr(vel, np.float64), _ptr(u, np.float64)]
    mem = _mem_of(*[a[1] for a in args])
    _check(lib().crk_set_state(sim, *[a[0] for a in args], ctypes.c_int(mem)))


def crk_get_sums(sim):
    mom = (ctypes.c_double * 3)()
    e = ctypes.c_double()
    nf = ctypes.c_int64()
    _check(lib().crk_get_sums(sim, mom, ctypes.byref(e), ctypes.byref(nf)))
    return list(mom), float(e.value), int(nf.value)


def crk_get_size(sim):
    n = ctypes.c_int64()
    nb = ctypes.c_int()
    _check(lib().crk_get_size(sim, ctypes.byref(n), ctypes.byref(nb)))
    return int(n.value), int(nb.value)


def crk_set_timing(sim, enable: bool):
    _check(lib().crk_set_timing(sim, ctypes.c_int(1 if enable else 0)))


def crk_get_timings(sim) -> dict:
    t = Timings()
    _check(lib().crk_get_timings(sim, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in Timings._fields_}


def crk_get_tree(sim) -> dict:
    """Leaves and leaf-pair lists of the handle's last tree, as host arrays:
    order (original index of each sorted position), leaf_start, leaf_count,
    leaf_species, leaf_centre (nleaf x 3), leaf_half (nleaf x 3), and the CSR
    lists hydro_row/hydro_col, grav_row/grav_col."""
    t = Tree()
    _check(lib().crk_get_tree(sim, ctypes.byref(t)))
    n, nl = int(t.n), int(t.nleaf)
    out = {"order": np.zeros(n, np.int64), "leaf_start": np.zeros(nl, np.uint32),
           "leaf_count": np.zeros(nl, np.uint32), "leaf_species": np.zeros(nl, np.uint8),
           "leaf_centre": np.zeros((nl, 3)), "leaf_half": np.zeros((nl, 3), np.float32),
           "hydro_row": np.zeros(nl + 1, np.uint32), "hydro_col": np.zeros(int(t.npair_hydro), np.uint32),
           "grav_row": np.zeros(nl + 1, np.uint32), "grav_col": np.zeros(int(t.npair_grav), np.uint32)}
    for k, v in out.items():
        setattr(t, k, v.ctypes.data if v.size else None)
    _check(lib().crk_get_tree(sim, ctypes.byref(t)))
    return out


def crk_fma_peak(precision: int, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (FP32 for
    CRK_MIXED, FP64 for CRK_FP64)."""
    out = ctypes.c_double()
    _check(lib().crk_fma_peak(ctypes.c_int(precision), ctypes.byref(out), _stream_handle(stream)))
    return float(out.value)


def crk_destroy(sim):
    _check(lib().crk_destroy(sim))


def crk_fof(sim, b: float, species_mask: int = 1, n: int | None = None):
    """Friends-of-friends groups (linking length b, species bits as in
    crk_fof); returns (group int64[N], number of groups)."""
    if n is None:
        n = crk_get_size(sim)[0]
    grp = np.zeros(n, np.int64)
    ng = ctypes.c_int64()
    _check(lib().crk_fof(sim, ctypes.c_double(b), ctypes.c_int(species_mask),
                         grp.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ng), ctypes.c_int(CRK_MEM_HOST)))
    return grp, int(ng.value)


def crk_pm_accel(sim, out=None):
    """Long-range mesh acceleration (N, 3) of the current state, load order
    (crk_pm_accel).  ``out``: a NumPy array or a CUDA tensor of 3N doubles;
    a new NumPy array when None."""
    if out is None:
        out = np.zeros((crk_get_size(sim)[0], 3))
    p, mem, keep = _ptr(out, np.float64)
    if mem == CRK_MEM_HOST and keep is not out:
        raise TypeError("out must be a contiguous float64 array")
    _check(lib().crk_pm_accel(sim, p, ctypes.c_int(mem)))
    return out


def crk_step_bins(sim, dt_long: float, depth: int, nlong: int = 1, eta: float = 0.025,
                  courant: float = 0.25):
    """Hierarchical time steps (crk_step_bins); returns the number of active
    particles of every substep (int64, nlong * 2^depth)."""
    counts = np.zeros((max(nlong, 0) << depth) if 0 <= depth <= 20 else 0, np.int64)
    _check(lib().crk_step_bins(sim, ctypes.c_double(dt_long), ctypes.c_int(depth), ctypes.c_int(nlong),
                               ctypes.c_double(eta), ctypes.c_double(courant),
                               counts.ctypes.data_as(ctypes.c_void_p)))
    return counts


def crk_get_bins(sim, n: int | None = None) -> np.ndarray:
    """Timestep bin of every particle, load order (crk_get_bins)."""
    if n is None:
        n = crk_get_size(sim)[0]
    out = np.zeros(n, np.uint8)
    _check(lib().crk_get_bins(sim, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(CRK_MEM_HOST)))
    return out


def crk_autotune(sim, caps=(32, 64, 128)):
    """Times one force evaluation per leaf capacity, keeps the fastest;
    returns (best capacity, {capacity: ms})."""
    arr = (ctypes.c_int * len(caps))(*caps)
    ms = (ctypes.c_double * len(caps))()
    best = ctypes.c_int()
    _check(lib().crk_autotune(sim, arr, ctypes.c_int(len(caps)), ctypes.byref(best), ms))
    return int(best.value), {c: float(m) for c, m in zip(caps, ms)}


def crk_autotune_ex(sim, caps=(32, 64, 128), forms=(0, 1, 2, 3)):
    """Times one force evaluation per (leaf capacity, pair decomposition: a bit
    set of CRK_GRAVITY_PAIRS_ONCE and CRK_HYDRO_PAIRS_ONCE), keeps the fastest;
    returns (best capacity, best form, {(capacity, form): ms})."""
    ca = (ctypes.c_int * len(caps))(*caps)
    fa = (ctypes.c_int * len(forms))(*forms)
    ms = (ctypes.c_double * (len(caps) * len(forms)))()
    bc, bf = ctypes.c_int(), ctypes.c_int()
    _check(lib().crk_autotune_ex(sim, ca, ctypes.c_int(len(caps)), fa, ctypes.c_int(len(forms)), ctypes.byref(bc),
                                 ctypes.byref(bf), ms))
    grid = {(c, f): float(ms[k * len(forms) + j]) for k, c in enumerate(caps) for j, f in enumerate(forms)}
    return int(bc.value), int(bf.value), grid


def crk_service_create(hbm_budget_bytes: int, max_slots: int, precision=CRK_MIXED, leaf_cap=64,
                       device=0, snapshot_every=0, size_classes=0, lane_priority=0) -> ctypes.c_void_p:
    p = ServiceParams()
    p.size_classes = size_classes
    p.lane_priority = lane_priority
    p.hbm_budget_bytes = int(hbm_budget_bytes)
    p.max_slots = max_slots
    p.precision = precision
    p.leaf_cap = leaf_cap
    p.device = device
    p.snapshot_every = snapshot_every
    h = ctypes.c_void_p()
    _check(lib().crk_service_create(ctypes.byref(p), ctypes.byref(h)))
    return h


def crk_submit(svc, phys: Physics, pos, vel, mass, u, h, species, dt: float, nsteps: int,
               resume=None) -> int:
    """Queues a job; `resume` (a snapshot dict from crk_service_snapshot, with
    the job's original mass, h and species) continues it from that state."""
    j = Job()
    j.phys = phys
    arrs = [np.ascontiguousarray(pos, np.float64), np.ascontiguousarray(vel, np.float64),
            np.ascontiguousarray(mass, np.float64), np.ascontiguousarray(u, np.float64),
            np.ascontiguousarray(h, np.float64), np.ascontiguousarray(species, np.uint8)]
    j.n = arrs[2].shape[0]
    for name, a in zip(("pos", "vel", "mass", "u", "h", "species"), arrs):
        setattr(j, name, a.ctypes.data_as(ctypes.c_void_p))
    if resume is not None:
        acc = np.ascontiguousarray(resume["acc"], np.float64)
        dudt = np.ascontiguousarray(resume["dudt"], np.float64)
        arrs += [acc, dudt]
        j.acc = acc.ctypes.data_as(ctypes.c_void_p)
        j.dudt = dudt.ctypes.data_as(ctypes.c_void_p)
        j.steps_done = int(resume["steps_done"])
    j.dt = dt
    j.nsteps = nsteps
    t = ctypes.c_uint64()
    _check(lib().crk_submit(svc, ctypes.byref(j), ctypes.byref(t)))
    return int(t.value)


def crk_poll(svc, ticket: int, n: int, timeout_us: int = -1, state: bool = True):
    """Returns None while pending, else a dict with the final state (unless
    state is False: latencies only, the state is not copied) and latencies
    (raises CrkError if the job failed)."""
    r = JobResult()
    out = {}
    if state:
        out = dict(pos=np.zeros((n, 3)), vel=np.zeros((n, 3)), u=np.zeros(n))
        r.pos = out["pos"].ctypes.data_as(ctypes.c_void_p)
        r.vel = out["vel"].ctypes.data_as(ctypes.c_void_p)
        r.u = out["u"].ctypes.data_as(ctypes.c_void_p)
    rc = lib().crk_poll(svc, ctypes.c_uint64(ticket), ctypes.byref(r), ctypes.c_int64(timeout_us))
    if rc == CRK_EPENDING:
        return None
    _check(rc)
    out.update(latency_ns=int(r.latency_ns), queue_ns=int(r.queue_ns))
    return out


def crk_service_destroy(svc):
    _check(lib().crk_service_destroy(svc))


def crk_service_snapshot(svc, ticket: int, n: int):
    """The job's latest complete snapshot (dict), or None if none was taken yet."""
    s = JobSnapshot()
    out = dict(pos=np.zeros((n, 3)), vel=np.zeros((n, 3)), u=np.zeros(n), acc=np.zeros((n, 3)),
               dudt=np.zeros(n))
    for k, v in out.items():
        setattr(s, k, v.ctypes.data_as(ctypes.c_void_p))
    rc = lib().crk_service_snapshot(svc, ctypes.c_uint64(ticket), ctypes.byref(s))
    if rc == CRK_EPENDING:
        return None
    _check(rc)
    out["steps_done"] = int(s.steps_done)
    return out


def crk_service_cancel(svc):
    _check(lib().crk_service_cancel(svc))


def crk_neighbours_noalloc(n: int, pos, h, species, box: float, count, hash_, stream=None) -> int:
    """Allocation-free hydro gather-set sizes and hashes (device tensors
    only).  Returns the C return code unchanged (the call does not update
    crk_last_error); work is queued on ``stream``."""
    args = [_ptr(pos, np.float64), _ptr(h, np.float64), _ptr(species, np.uint8),
            _ptr(count, np.int32), _ptr(hash_, np.uint64)]
    if any(a[1] != CRK_MEM_DEVICE for a in args):
        raise TypeError("crk_neighbours_noalloc takes CUDA device tensors")
    return int(lib().crk_neighbours_noalloc(ctypes.c_int64(n), *[a[0] for a in args[:3]],
                                            ctypes.c_double(box), args[3][0], args[4][0],
                                            _stream_handle(stream)))


def crk_last_error() -> str:
    return lib().crk_last_error().decode()


# ------------------------------------------------------- convenience class
class Sim:
    """Owns one crk_sim handle (create / load / forces / step / destroy)."""

    def __init__(self, phys: Physics | None = None, leaf_cap=64, precision=CRK_MIXED, cm_level=0,
                 stream=None, rebuild_every=1, pm_grid=0, flags=0, graph_margin_pct=0):
        self.handle = crk_create(params(phys, leaf_cap, precision, cm_level, rebuild_every=rebuild_every,
                                        pm_grid=pm_grid, flags=flags, graph_margin_pct=graph_margin_pct),
                                 stream)

    def load(self, box):
        crk_load(self.handle, box.pos, box.vel, box.mass, box.u, box.h, box.species)
        self.n = box.n
        return self

    def forces(self, counts=True):
        n = self.n
        outs = dict(acc=np.zeros((n, 3)), dudt=np.zeros(n), rho=np.zeros(n), A=np.zeros(n),
                    B=np.zeros((n, 3)), gradA=np.zeros((n, 3)), gradB=np.zeros((n, 3, 3)))
        if counts:
            outs.update(nbr_count=np.zeros(n, np.int32), nbr_hash=np.zeros(n, np.uint64),
                        grav_count=np.zeros(n, np.int32), grav_hash=np.zeros(n, np.uint64))
        mom, e = crk_forces(self.handle, **outs)
        outs["momentum_rate"] = np.array(mom)
        outs["energy_rate"] = e
        return outs

    def step(self, dt, nsteps=1):
        crk_step(self.handle, dt, nsteps)

    def state(self):
        n = crk_get_size(self.handle)[0]
        pos, vel, u = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
        crk_get_state(self.handle, pos, vel, u)
        return pos, vel, u

    def close(self):
        if self.handle:
            crk_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def box_physics(box) -> Physics:
    """Physics of a ``workloads.Box``."""
    return physics(**box.params())
