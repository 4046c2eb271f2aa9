"""Hierarchical (block) time steps: plain FP64 numpy around the oracle's forces.

TEST INFRASTRUCTURE.  Only the test suite loads this module; the product
path never calls it and shares no code with it.

The paper integrates the short-range physics with particles grouped into
power-of-two timestep bins that follow local conditions, evaluating forces
only where a particle's step ends (Sec. II and IV-B1: adaptive integration
after Saitoh & Makino 2010; only active leaves are updated in a substep).
It prints no formula, so this module fixes the reading:

* A long step D_t is cut into 2^depth substeps of d = D_t / 2^depth.  A
  particle in bin b (0 <= b <= depth) takes steps of dt_b = D_t / 2^b, that
  is L_b = 2^(depth - b) substeps; its steps start at multiples of L_b.
* Substep s (0 <= s < 2^depth), in this order:
    1. opening kick of every particle whose step starts at s:
       v += dt_b/2 a, u += dt_b/2 du (gas u floored);
    2. drift of every particle: x = wrap(x + d v);
    3. forces at t_(s+1) for every particle whose step ends at s + 1 (the
       active ones), with every particle's predicted v^ = v + tau a and
       u^ = max(u + tau du, u_floor) (gas), tau = ((s + 1 - s0) - L_b / 2) d
       where s0 is the start of its current step (tau = dt_b / 2 for an
       active particle, as in the fixed-step form);
    4. closing kick of the active particles with the new a, du (u floored);
    5. a new bin for every active particle: the shallowest b with
       D_t / 2^b <= min(dt_acc, dt_cfl), at most depth, where
       dt_acc = sqrt(2 eta eps / |a|) (not applied when eps = 0 or a = 0) and
       dt_cfl = courant h / c with c = sqrt(gamma (gamma - 1) u) (gas with
       u > 0); a particle may only move to a bin whose steps start at s + 1,
       so b = max(b_new, depth - trailing_zeros(s + 1)) (0 at the end of the
       long step).
* Before the first long step with no stored forces every particle gets its
  forces at t = 0 and a bin from the same criterion.
* With a long-range mesh (pm_grid > 0; Sec. IV-A: the long-range force is
  integrated with the long PM step, the short-range physics in the substeps):
  every long step is wrapped in two half kicks v += D_t/2 a_mesh(x), the mesh
  acceleration of ``oracle.pm`` at the positions of its start and of its end;
  the substeps and the bin criterion see the short-range and hydro forces
  only, and the forces stored at the start are recomputed (short-range only).

With depth = 0 this is the fixed-step KDK of ``oracle.kdk``; with every
particle in the deepest bin it is that KDK at dt = D_t / 2^depth.
"""
from __future__ import annotations

import math

import numpy as np

from . import forces as _forces
from . import pm as _pm


def _wrap(x: np.ndarray, L: float) -> np.ndarray:
    """Position wrap into [0, L) after a drift (x + d v moved by at most L)."""
    x = np.where(x >= L, x - L, x)
    neg = x < 0.0
    x = np.where(neg, x + L, x)
    return np.where(neg & (x >= L), 0.0, x)


def _floor(u: np.ndarray, gas: np.ndarray, fl: float) -> tuple[np.ndarray, int]:
    low = gas & (u < fl)
    return np.where(low, fl, u), int(low.sum())


def new_bins(acc, u, h, gas, params, dt_long: float, depth: int, eta: float, courant: float,
             b_sync: int) -> np.ndarray:
    """Step 5: the bin of every particle from its acceleration and (gas) u."""
    n = len(h)
    ax, ay, az = acc[:, 0], acc[:, 1], acc[:, 2]
    amag = np.sqrt((ax * ax + ay * ay) + az * az)
    dt = np.full(n, np.inf)
    if params.eps_soft > 0.0:
        num = (2.0 * eta) * params.eps_soft
        with np.errstate(divide="ignore"):
            da = np.where(amag > 0.0, np.sqrt(num / np.where(amag > 0.0, amag, 1.0)), np.inf)
        dt = np.minimum(dt, da)
    g = params.gamma * (params.gamma - 1.0)
    hot = gas & (u > 0.0)
    c = np.sqrt(g * np.where(hot, u, 1.0))
    dc = np.where(hot, (courant * h) / c, np.inf)
    dt = np.minimum(dt, dc)
    b = np.zeros(n, np.int64)
    for k in range(depth):
        # still too long: D_t / 2^b > dt
        b = np.where(math.ldexp(dt_long, -k) > dt, k + 1, b)
    return np.maximum(b, b_sync)


def kdk_bins(pos, vel, mass, u, h, species, params, dt_long: float, depth: int, nlong: int,
             eta: float, courant: float, acc=None, dudt=None, bins=None, pm_grid: int = 0) -> dict:
    """Run nlong long steps; returns the final pos, vel, u, acc, dudt, bins,
    the floor events and the number of active particles of every substep."""
    pos = np.array(pos, np.float64).reshape(-1, 3)
    vel = np.array(vel, np.float64).reshape(-1, 3)
    u = np.array(u, np.float64).copy()
    mass = np.asarray(mass, np.float64)
    h = np.asarray(h, np.float64)
    sp = np.asarray(species, np.uint8)
    gas = sp == 1
    n = len(mass)
    L = params.L
    nfloor = 0
    nsub = 1 << depth
    d = math.ldexp(dt_long, -depth)
    mesh = (lambda x: _pm.accelerations(x, mass, L, pm_grid, params.G, params.r_split)) if pm_grid else None
    if acc is None or mesh is not None:
        r = _forces(pos, vel, mass, u, h, sp, params)
        if r["rc"]:
            raise RuntimeError(f"oracle forces failed: {r['rc']}")
        acc, dudt = r["acc"].copy(), r["dudt"].copy()
        bins = new_bins(acc, u, h, gas, params, dt_long, depth, eta, courant, 0)
    else:
        acc = np.array(acc, np.float64).reshape(-1, 3)
        dudt = np.array(dudt, np.float64).copy()
        bins = np.asarray(bins, np.int64).copy()
    active_counts = []
    for _ in range(nlong):
        if mesh is not None:
            vel = vel + (0.5 * dt_long) * mesh(pos)
        for s in range(nsub):
            Lb = np.left_shift(1, depth - bins)          # substeps per step
            hdt = Lb * (0.5 * d)                          # dt_b / 2, exact
            opening = (s % Lb) == 0
            vel = np.where(opening[:, None], vel + hdt[:, None] * acc, vel)
            u = np.where(opening, u + hdt * dudt, u)
            u, k = _floor(u, gas & opening, params.u_floor)
            nfloor += k
            pos = _wrap(pos + d * vel, L)
            s0 = (s // Lb) * Lb
            tau = (2 * (s + 1 - s0) - Lb) * (0.5 * d)
            vp = vel + tau[:, None] * acc
            up, k = _floor(u + tau * dudt, gas, params.u_floor)
            nfloor += k
            active = ((s + 1) % Lb) == 0
            active_counts.append(int(active.sum()))
            r = _forces(pos, vp, mass, up, h, sp, params)
            if r["rc"]:
                raise RuntimeError(f"oracle forces failed: {r['rc']}")
            acc = np.where(active[:, None], r["acc"], acc)
            dudt = np.where(active, r["dudt"], dudt)
            vel = np.where(active[:, None], vel + hdt[:, None] * acc, vel)
            u = np.where(active, u + hdt * dudt, u)
            u, k = _floor(u, gas & active, params.u_floor)
            nfloor += k
            t = s + 1
            b_sync = 0 if t == nsub else depth - ((t & -t).bit_length() - 1)
            nb = new_bins(acc, u, h, gas, params, dt_long, depth, eta, courant, b_sync)
            bins = np.where(active, nb, bins)
        if mesh is not None:
            vel = vel + (0.5 * dt_long) * mesh(pos)
    return dict(pos=pos, vel=vel, u=u, acc=acc, dudt=dudt, bins=bins, nfloor=nfloor,
                active_counts=np.array(active_counts, np.int64))
