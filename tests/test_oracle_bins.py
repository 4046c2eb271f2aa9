"""Pins of the oracle's hierarchical time steps (``oracle.bins``) against what
fixes them from outside: the oracle's own fixed-step KDK in C in the two
cases that reduce to it (one bin of depth 0; every particle in the deepest
bin), two non-interacting groups in different bins that must each follow
their own fixed-step run, the bin criterion by hand, and second-order
convergence to a fine fixed-step run when particles of different bins
interact (a predictor that ignored the inactive particles' accelerations
would drop it to first order)."""
import math

import numpy as np
import pytest

import oracle
from oracle import bins as ob
from paper_2510_03557_gb300 import workloads as wl


def _box(n=12, seed=4):
    box = wl.gaussian_field_box(n, seed=seed)
    box.vel = box.vel * 20.0
    return box, oracle.make_params(**box.params())


def test_depth_zero_is_the_fixed_step_kdk():
    box, op = _box()
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, 1e-3, 3)
    got = ob.kdk_bins(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, 1e-3, 0, 3,
                      eta=0.025, courant=0.25)
    for k in ("pos", "vel", "u", "acc", "dudt"):
        assert np.array_equal(got[k], ref[k]), k
    assert got["nfloor"] == ref["nfloor"]
    assert np.all(got["bins"] == 0) and list(got["active_counts"]) == [box.n] * 3


def test_every_particle_in_the_deepest_bin_is_the_fixed_step_kdk_at_the_substep():
    box, op = _box()
    depth, dt_long = 3, 2e-3
    # a tiny Courant factor and eta put every particle in the deepest bin
    got = ob.kdk_bins(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, dt_long, depth, 1,
                      eta=1e-12, courant=1e-12)
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, dt_long / 8, 8)
    assert np.all(got["bins"] == depth)
    for k in ("pos", "vel", "u", "acc", "dudt"):
        assert np.array_equal(got[k], ref[k]), k


def _blob(centre, n, spacing, u):
    g = (np.arange(n) - (n - 1) / 2) * spacing
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + np.asarray(centre)
    m = len(pos)
    return pos, np.full(m, u)


def test_separated_groups_follow_their_own_fixed_steps():
    """A hot blob in the deepest bin and a cold one in bin 0, far apart (no
    pair within r_cut or H): each is the fixed-step KDK at its own dt."""
    sp_, n1 = 0.02, 3
    # Courant 0.05 h / c: 3.5e-4 for the hot blob (bin 3: 2.5e-4 <= dt < 5e-4),
    # 0.02 for the cold one (bin 0)
    pa, ua = _blob([0.25, 0.25, 0.25], n1, sp_, 7.35)
    pb, ub = _blob([0.75, 0.75, 0.75], n1, sp_, 0.00225)
    pos = np.concatenate([pa, pb])
    u = np.concatenate([ua, ub])
    n = len(pos)
    rng = np.random.default_rng(7)
    pos = pos + rng.uniform(-0.002, 0.002, pos.shape)
    vel = rng.normal(0.0, 0.3, (n, 3))
    mass = np.full(n, 1e-5)
    h = np.full(n, 0.02)
    sp = np.ones(n, np.uint8)
    op = oracle.make_params(box=1.0, G=1.0, r_cut=0.1, r_split=0.02, eps_soft=0.0)
    depth, dt_long = 3, 2e-3
    got = ob.kdk_bins(pos, vel, mass, u, h, sp, op, dt_long, depth, 1, eta=0.025, courant=0.05)
    na = len(pa)
    assert np.all(got["bins"][:na] == 3) and np.all(got["bins"][na:] == 0)
    assert list(got["active_counts"]) == [na] * 7 + [n]
    A = slice(0, na)
    B = slice(na, n)
    ra = oracle.kdk(pos[A], vel[A], mass[A], u[A], h[A], sp[A], op, dt_long / 8, 8)
    rb = oracle.kdk(pos[B], vel[B], mass[B], u[B], h[B], sp[B], op, dt_long, 1)
    for k in ("pos", "vel", "u"):
        assert np.array_equal(got[k][A], ra[k]), k
        # B drifts in 8 substeps instead of one step: equal to rounding
        assert np.allclose(got[k][B], rb[k], rtol=1e-13, atol=1e-15), k


def test_bin_criterion_by_hand():
    op = oracle.make_params(box=1.0, gamma=5.0 / 3.0, eps_soft=0.01)
    acc = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0], [300.0, 0.0, 400.0], [0.0, 0.0, 0.0]])
    u = np.array([0.0, 0.0, 0.0, 9.0])
    h = np.array([0.0, 0.0, 0.0, 0.05])
    gas = np.array([False, False, False, True])
    eta, courant, dt_long, depth = 0.025, 0.25, 0.1, 6
    b = ob.new_bins(acc, u, h, gas, op, dt_long, depth, eta, courant, 0)
    # |a| = 5: dt = sqrt(2 * 0.025 * 0.01 / 5) = 0.01 -> 0.1 / 2^4 = 0.00625 <= 0.01 < 0.0125
    # |a| = 500: dt = 0.001 -> 0.1 / 2^7 would be needed: capped at depth 6
    # gas: c = sqrt(10/9 * 9) = sqrt(10), dt = 0.0125 / sqrt(10) = 0.00395 -> 2^5: 0.003125
    assert list(b) == [0, 4, 6, 5]
    # a particle may only move to a bin whose steps start now
    assert list(ob.new_bins(acc, u, h, gas, op, dt_long, depth, eta, courant, 5)) == [5, 5, 6, 5]


def test_mixed_bins_converge_at_second_order():
    """A compressing gas blob with a hot core (bin 2) and a cold envelope
    (bin 0) that interact, against a fine fixed-step run: halving the long
    step (Courant factor halved with it, so the bins stay) divides the error
    by about 4.  A predictor that took every particle as if its step ended
    now (tau = dt_b / 2 for the inactive ones too) converges at first order
    here (ratios 2.5 and 2.2)."""
    rng = np.random.default_rng(11)
    pos, u = _blob([0.5, 0.5, 0.5], 6, 0.02, 1.0)
    r = np.linalg.norm(pos - 0.5, axis=1)
    u = np.where(r < 0.035, 40.0, 1.0)
    pos = pos + rng.uniform(-0.002, 0.002, pos.shape)
    n = len(pos)
    vel = -3.0 * (pos - 0.5)
    mass = np.full(n, 1e-5)
    h = np.full(n, 0.025)
    sp = np.ones(n, np.uint8)
    op = oracle.make_params(box=1.0, G=0.0, r_cut=0.1, r_split=0.02, eps_soft=0.0)
    T, depth = 4e-3, 2
    ref = oracle.kdk(pos, vel, mass, u, h, sp, op, T / 1024, 1024)
    hot = u > 10.0
    errs = []
    for k in (4, 8, 16):
        got = ob.kdk_bins(pos, vel, mass, u, h, sp, op, T / k, depth, k, eta=0.025, courant=0.4 / k)
        assert np.all(got["bins"][hot] == 2) and np.all(got["bins"][~hot] == 0)
        assert list(got["active_counts"][:4]) == [int(hot.sum())] * 3 + [n]
        errs.append(np.linalg.norm(got["vel"] - ref["vel"]))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(3.2 < q < 5.0 for q in ratios), (errs, ratios)


def test_mesh_long_step_is_a_leapfrog_when_nothing_is_near():
    """Dark matter far apart (no pair within r_cut) feels only the mesh: the
    long step with its two mesh half kicks and the substeps (bin 0: drifts
    only) is the textbook leapfrog at dt = D_t with the mesh force."""
    from oracle import pm

    rng = np.random.default_rng(21)
    g = np.arange(4) * 0.25 + 0.125
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = pos + rng.uniform(-0.02, 0.02, pos.shape)
    n = len(pos)
    vel = rng.normal(0.0, 0.05, (n, 3))
    mass = rng.uniform(0.5, 1.5, n)
    zero = np.zeros(n)
    sp = np.zeros(n, np.uint8)
    op = oracle.make_params(box=1.0, G=1.0, r_cut=0.05, r_split=0.05, eps_soft=0.001)
    dt, nlong, ng = 2e-3, 3, 16
    x, v = pos.copy(), vel.copy()
    for _ in range(nlong):
        v = v + (0.5 * dt) * pm.accelerations(x, mass, 1.0, ng, 1.0, 0.05)
        x = x + dt * v
        x = np.where(x >= 1.0, x - 1.0, x)
        x = np.where(x < 0.0, x + 1.0, x)
        v = v + (0.5 * dt) * pm.accelerations(x, mass, 1.0, ng, 1.0, 0.05)
    got = ob.kdk_bins(pos, vel, mass, zero, zero, sp, op, dt, 0, nlong, eta=0.025, courant=0.25, pm_grid=ng)
    assert np.array_equal(got["pos"], x)
    assert np.array_equal(got["vel"], v)
    # deeper bins change nothing but the drift, cut into four substeps
    got = ob.kdk_bins(pos, vel, mass, zero, zero, sp, op, dt, 2, nlong, eta=0.025, courant=0.25, pm_grid=ng)
    assert np.all(got["bins"] == 0)
    assert np.allclose(got["pos"], x, rtol=0, atol=1e-14)
    assert np.allclose(got["vel"], v, rtol=1e-12, atol=0)
