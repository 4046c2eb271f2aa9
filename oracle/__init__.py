"""CPU FP64 oracle for the CRKSPH + short-range gravity pair solver.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code
with the CUDA library: its C source (``crk_oracle.c``) is compiled on its own
with ``gcc -O2 -fopenmp -ffp-contract=off`` and loaded here with ctypes.

Every function follows the plain definitions of the method (paper Sec. IV-A
and Eq. 1-2, with the readings listed in the C file's header) and is pinned by
the ``-m "not gpu"`` oracle tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crk_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcrk_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ESINGULAR = -5


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libcrk_oracle.so``."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("G", ctypes.c_double), ("gamma", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("r_split", ctypes.c_double),
                ("eps_soft", ctypes.c_double), ("av_alpha", ctypes.c_double),
                ("av_beta", ctypes.c_double), ("av_eps2", ctypes.c_double),
                ("u_floor", ctypes.c_double), ("brute", ctypes.c_int),
                ("nthreads", ctypes.c_int)]


def make_params(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.0, r_split=1.0, eps_soft=0.0,
                av_alpha=1.0, av_beta=2.0, av_eps2=0.01, u_floor=1e-10, brute=False,
                nthreads=0) -> Params:
    return Params(box, G, gamma, r_cut, r_split, eps_soft, av_alpha, av_beta, av_eps2,
                  u_floor, int(bool(brute)), int(nthreads))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d = ctypes.c_double
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.orc_W.restype = d
            L.orc_W.argtypes = [d, d]
            L.orc_gradW_factor.restype = d
            L.orc_gradW_factor.argtypes = [d, d]
            L.orc_S.restype = d
            L.orc_S.argtypes = [d, d]
            for name in ("orc_neighbours", "orc_expand_mask", "orc_density", "orc_moments",
                         "orc_corrections", "orc_hydro", "orc_gravity", "orc_pair_forces",
                         "orc_crk_identities", "orc_forces", "orc_kdk", "orc_fof"):
                getattr(L, name).restype = ctypes.c_int
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def W(r, h):
    return lib().orc_W(float(r), float(h))


def gradW_factor(r, h):
    return lib().orc_gradW_factor(float(r), float(h))


def S(r, r_s):
    return lib().orc_S(float(r), float(r_s))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def neighbours(pos, h, species, params: Params, kind: int):
    """kind 0: hydro gather set, 1: hydro pair set, 2: gravity set.
    Returns (count int32[N], hash uint64[N]) of original indices."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    h = _f64(h)
    sp = _u8(species)
    cnt = np.zeros(n, np.int32)
    hs = np.zeros(n, np.uint64)
    rc = lib().orc_neighbours(ctypes.c_int64(n), _p(pos), _p(h), _p(sp), ctypes.byref(params),
                              ctypes.c_int(kind), _p(cnt), _p(hs))
    if rc:
        raise RuntimeError(f"orc_neighbours failed: {rc}")
    return cnt, hs


def fof(pos, species, box: float, b: float, species_mask: int = 1):
    """Friends-of-friends groups (in situ halo finding, Sec. IV-B3): particles
    of the species in `species_mask` (bit 0 DM, bit 1 gas) linked when
    r < b; returns (group int64[N]: the smallest index of the particle's
    group, -1 for other species; number of groups)."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    grp = np.zeros(n, np.int64)
    ng = ctypes.c_int64()
    rc = lib().orc_fof(ctypes.c_int64(n), _p(pos), _p(_u8(species)), ctypes.c_double(box),
                       ctypes.c_double(b), ctypes.c_int(species_mask), _p(grp), ctypes.byref(ng))
    if rc:
        raise RuntimeError(f"orc_fof failed: {rc}")
    return grp, int(ng.value)


def expand_mask(pos, h, species, params: Params, mask):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    out = np.zeros(n, np.uint8)
    rc = lib().orc_expand_mask(ctypes.c_int64(n), _p(pos), _p(_f64(h)), _p(_u8(species)),
                               ctypes.byref(params), _p(_u8(mask)), _p(out))
    if rc:
        raise RuntimeError(f"orc_expand_mask failed: {rc}")
    return out


def density(pos, mass, u, h, species, params: Params, mask=None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    rho, V, P, c = (np.zeros(n) for _ in range(4))
    rc = lib().orc_density(ctypes.c_int64(n), _p(pos), _p(_f64(mass)), _p(_f64(u)), _p(_f64(h)),
                           _p(_u8(species)), ctypes.byref(params),
                           _p(None if mask is None else _u8(mask)),
                           _p(rho), _p(V), _p(P), _p(c))
    if rc:
        raise RuntimeError(f"orc_density failed: {rc}")
    return rho, V, P, c


def moments(pos, V, h, species, params: Params, mask=None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    mom = np.zeros((n, 40))
    rc = lib().orc_moments(ctypes.c_int64(n), _p(pos), _p(_f64(V)), _p(_f64(h)), _p(_u8(species)),
                           ctypes.byref(params), _p(None if mask is None else _u8(mask)), _p(mom))
    if rc:
        raise RuntimeError(f"orc_moments failed: {rc}")
    return mom


def corrections(mom, species, mask=None):
    mom = _f64(mom, (-1, 40))
    n = mom.shape[0]
    A = np.zeros(n)
    B = np.zeros((n, 3))
    dA = np.zeros((n, 3))
    dB = np.zeros((n, 3, 3))
    bad = ctypes.c_int64(-1)
    rc = lib().orc_corrections(ctypes.c_int64(n), _p(mom), _p(_u8(species)),
                               _p(None if mask is None else _u8(mask)),
                               _p(A), _p(B), _p(dA), _p(dB), ctypes.byref(bad))
    return rc, int(bad.value), A, B, dA, dB


def hydro(pos, vel, mass, h, species, rho, V, P, c, A, B, dA, dB, params: Params, mask=None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    acc = np.zeros((n, 3))
    dudt = np.zeros(n)
    rc = lib().orc_hydro(ctypes.c_int64(n), _p(pos), _p(_f64(vel, (-1, 3))), _p(_f64(mass)),
                         _p(_f64(h)), _p(_u8(species)), _p(_f64(rho)), _p(_f64(V)), _p(_f64(P)),
                         _p(_f64(c)), _p(_f64(A)), _p(_f64(B, (-1, 3))), _p(_f64(dA, (-1, 3))),
                         _p(_f64(dB, (-1, 3, 3))), ctypes.byref(params),
                         _p(None if mask is None else _u8(mask)), _p(acc), _p(dudt))
    if rc:
        raise RuntimeError(f"orc_hydro failed: {rc}")
    return acc, dudt


def gravity(pos, mass, species, params: Params, mask=None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    acc = np.zeros((n, 3))
    rc = lib().orc_gravity(ctypes.c_int64(n), _p(pos), _p(_f64(mass)), _p(_u8(species)),
                           ctypes.byref(params), _p(None if mask is None else _u8(mask)), _p(acc))
    if rc:
        raise RuntimeError(f"orc_gravity failed: {rc}")
    return acc


def pair_forces(state: dict, params: Params, i: int, j: int):
    """Hydro and gravity force on i from j for one pair (uses the arrays of
    ``forces``' result plus the inputs)."""
    s = state
    Fh = np.zeros(3)
    Fg = np.zeros(3)
    pos = _f64(s["pos"], (-1, 3))
    rc = lib().orc_pair_forces(ctypes.c_int64(pos.shape[0]), _p(pos), _p(_f64(s["vel"], (-1, 3))),
                               _p(_f64(s["mass"])), _p(_f64(s["h"])), _p(_u8(s["species"])),
                               _p(_f64(s["rho"])), _p(_f64(s["V"])), _p(_f64(s["P"])),
                               _p(_f64(s["c"])), _p(_f64(s["A"])), _p(_f64(s["B"], (-1, 3))),
                               _p(_f64(s["dA"], (-1, 3))), _p(_f64(s["dB"], (-1, 3, 3))),
                               ctypes.byref(params), ctypes.c_int64(i), ctypes.c_int64(j),
                               _p(Fh), _p(Fg))
    if rc:
        raise RuntimeError(f"orc_pair_forces failed: {rc}")
    return Fh, Fg


def crk_identities(pos, V, h, species, A, B, dA, dB, params: Params, mask=None):
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    out = np.zeros((n, 16))
    rc = lib().orc_crk_identities(ctypes.c_int64(n), _p(pos), _p(_f64(V)), _p(_f64(h)),
                                  _p(_u8(species)), _p(_f64(A)), _p(_f64(B, (-1, 3))),
                                  _p(_f64(dA, (-1, 3))), _p(_f64(dB, (-1, 3, 3))),
                                  ctypes.byref(params), _p(None if mask is None else _u8(mask)),
                                  _p(out))
    if rc:
        raise RuntimeError(f"orc_crk_identities failed: {rc}")
    return out


def forces(pos, vel, mass, u, h, species, params: Params, sample=None):
    """All passes.  With ``sample`` (indices), only the sampled particles'
    outputs are guaranteed (the masks are expanded so that every quantity
    they depend on is computed).  Returns a dict of arrays in input order."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    vel = _f64(vel, (-1, 3))
    mass, u, h = _f64(mass), _f64(u), _f64(h)
    sp = _u8(species)
    mh = mm = md = None
    if sample is not None:
        mh = np.zeros(n, np.uint8)
        mh[np.asarray(sample, dtype=np.int64)] = 1
        mm = expand_mask(pos, h, sp, params, mh)
        md = expand_mask(pos, h, sp, params, mm)
    out = dict(acc=np.zeros((n, 3)), dudt=np.zeros(n), rho=np.zeros(n), V=np.zeros(n),
               P=np.zeros(n), c=np.zeros(n), mom=np.zeros((n, 40)), A=np.zeros(n),
               B=np.zeros((n, 3)), dA=np.zeros((n, 3)), dB=np.zeros((n, 3, 3)))
    bad = ctypes.c_int64(-1)
    rc = lib().orc_forces(ctypes.c_int64(n), _p(pos), _p(vel), _p(mass), _p(u), _p(h), _p(sp),
                          ctypes.byref(params), _p(mh), _p(mm), _p(md),
                          *[_p(out[k]) for k in ("acc", "dudt", "rho", "V", "P", "c", "mom", "A",
                                                   "B", "dA", "dB")],
                          ctypes.byref(bad))
    out["rc"] = rc
    out["bad"] = int(bad.value)
    out.update(pos=pos, vel=vel, mass=mass, u=u, h=h, species=sp)
    return out


def kdk(pos, vel, mass, u, h, species, params: Params, dt: float, nsteps: int,
        acc=None, dudt=None):
    """Run nsteps KDK steps on copies of the state; returns a dict with the
    final pos, vel, u, acc, dudt and the number of floor events."""
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    u = _f64(u).copy()
    n = pos.shape[0]
    have = acc is not None
    acc = np.zeros((n, 3)) if acc is None else _f64(acc, (-1, 3)).copy()
    dudt = np.zeros(n) if dudt is None else _f64(dudt).copy()
    nfl = ctypes.c_int64(0)
    rc = lib().orc_kdk(ctypes.c_int64(n), _p(pos), _p(vel), _p(_f64(mass)), _p(u), _p(_f64(h)),
                       _p(_u8(species)), ctypes.byref(params), ctypes.c_double(dt),
                       ctypes.c_int(nsteps), _p(acc), _p(dudt), ctypes.c_int(int(have)),
                       ctypes.byref(nfl))
    if rc:
        raise RuntimeError(f"orc_kdk failed: {rc}")
    return dict(pos=pos, vel=vel, u=u, acc=acc, dudt=dudt, nfloor=int(nfl.value))
