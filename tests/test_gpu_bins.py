"""GPU parity of the hierarchical time steps (``crk_step_bins``) against the
oracle's ``oracle.bins.kdk_bins``, through the C ABI.

Bins and per-substep active counts are integers decided in FP64 on both
sides: equal in the FP64 form.  Positions, velocities and u: relative L2
1e-10 (FP64) or 2e-4 (mixed form, where a bin decision may differ for a
particle whose step size sits at a bin edge to FP32 rounding).
"""
import numpy as np
import pytest

import oracle
from oracle import bins as ob
from paper_2510_03557_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crk():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2510_03557_gb300 import crk as c

    return c


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def disp_err(pos, ref, pos0, L):
    d = pos - ref
    d = np.where(d > 0.5 * L, d - L, d)
    d = np.where(d < -0.5 * L, d + L, d)
    return np.linalg.norm(d) / np.linalg.norm(ref - pos0)


def _box():
    box = wl.gaussian_field_box(12, seed=4)
    box.vel = box.vel * 20.0
    return box


ETA, COURANT, DT_LONG, DEPTH = 0.01, 0.25, 8e-3, 3


@pytest.fixture(scope="module")
def reference():
    box = _box()
    op = oracle.make_params(**box.params())
    return box, ob.kdk_bins(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, DT_LONG, DEPTH, 2,
                            eta=ETA, courant=COURANT)


@pytest.mark.parametrize("leaf_cap", [32, 128])
def test_bins_fp64_match_oracle(crk, reference, leaf_cap):
    box, ref = reference
    assert len(np.unique(ref["bins"])) >= 3          # the case mixes bins
    with crk.Sim(crk.box_physics(box), leaf_cap=leaf_cap, precision=0) as sim:
        sim.load(box)
        counts = crk.crk_step_bins(sim.handle, DT_LONG, DEPTH, 2, ETA, COURANT)
        bins = crk.crk_get_bins(sim.handle)
        pos, vel, u = sim.state()
        _, _, nfloor = crk.crk_get_sums(sim.handle)
    assert np.array_equal(counts, ref["active_counts"])
    assert np.array_equal(bins, ref["bins"])
    assert disp_err(pos, ref["pos"], box.pos, box.L) <= 1e-10
    assert rel_l2(vel, ref["vel"]) <= 1e-10
    assert rel_l2(u, ref["u"]) <= 1e-10
    assert nfloor == ref["nfloor"]


def test_bins_mixed_match_oracle(crk, reference):
    box, ref = reference
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=1) as sim:
        sim.load(box)
        crk.crk_step_bins(sim.handle, DT_LONG, DEPTH, 2, ETA, COURANT)
        bins = crk.crk_get_bins(sim.handle)
        pos, vel, u = sim.state()
    assert np.mean(bins == ref["bins"]) >= 0.99
    assert disp_err(pos, ref["pos"], box.pos, box.L) <= 2e-4
    assert rel_l2(vel, ref["vel"]) <= 2e-4
    assert rel_l2(u, ref["u"]) <= 2e-4


def test_depth_zero_is_crk_step(crk):
    box = _box()
    # host-sized steps on both sides (the hierarchical steps are host-sized)
    flags = crk.CRK_FLAG_NO_GRAPH
    with crk.Sim(crk.box_physics(box), precision=1, flags=flags) as a, \
            crk.Sim(crk.box_physics(box), precision=1, flags=flags) as b:
        a.load(box)
        b.load(box)
        counts = crk.crk_step_bins(a.handle, 1e-3, 0, 3, ETA, COURANT)
        b.step(1e-3, 3)
        sa, sb = a.state(), b.state()
    assert list(counts) == [box.n] * 3
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)


def test_separated_groups_in_different_bins(crk):
    """The oracle pin's case on the GPU: a hot blob in the deepest bin and a
    cold one in bin 0, far apart."""
    g = (np.arange(3) - 1) * 0.02
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    blob = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos = np.concatenate([blob + 0.25, blob + 0.75])
    n = len(pos)
    rng = np.random.default_rng(7)
    pos = pos + rng.uniform(-0.002, 0.002, pos.shape)
    vel = rng.normal(0.0, 0.3, (n, 3))
    u = np.concatenate([np.full(27, 7.35), np.full(27, 0.00225)])
    mass, h, sp = np.full(n, 1e-5), np.full(n, 0.02), np.ones(n, np.uint8)
    op = oracle.make_params(box=1.0, G=1.0, r_cut=0.1, r_split=0.02, eps_soft=0.0)
    ref = ob.kdk_bins(pos, vel, mass, u, h, sp, op, 2e-3, 3, 1, eta=0.025, courant=0.05)
    phys = crk.physics(box=1.0, G=1.0, r_cut=0.1, r_split=0.02, eps_soft=0.0)
    with crk.Sim(phys, precision=0) as sim:
        crk.crk_load(sim.handle, pos, vel, mass, u, h, sp)
        counts = crk.crk_step_bins(sim.handle, 2e-3, 3, 1, 0.025, 0.05)
        bins = crk.crk_get_bins(sim.handle)
        gpos, gvel, gu = sim.state()
    assert list(counts) == [27] * 7 + [54]
    assert np.array_equal(bins, ref["bins"])
    assert np.allclose(gpos, ref["pos"], rtol=1e-12, atol=1e-15)
    assert rel_l2(gvel, ref["vel"]) <= 1e-10
    assert rel_l2(gu, ref["u"]) <= 1e-10


def test_bins_argument_errors(crk):
    box = _box()
    with crk.Sim(crk.box_physics(box)) as sim:
        sim.load(box)
        for args in ((0.0, 2, 1, ETA, COURANT), (1e-3, -1, 1, ETA, COURANT), (1e-3, 21, 1, ETA, COURANT),
                     (1e-3, 2, -1, ETA, COURANT), (1e-3, 2, 1, 0.0, COURANT), (1e-3, 2, 1, ETA, -1.0)):
            with pytest.raises(crk.CrkError) as e:
                crk.crk_step_bins(sim.handle, *args)
            assert e.value.code == crk.CRK_EINVAL


def test_batched_boxes_step_as_they_do_alone(crk):
    """Hierarchical steps of two boxes in one handle: each box ends exactly
    where it ends alone (boxes never interact, every box sorts all key bits
    and its active sets, lists and sums are its own)."""
    b1 = _box()
    b2 = wl.gaussian_field_box(10, seed=8)
    b2.vel = b2.vel * 20.0
    boxes = [b1, b2]
    cat = lambda k: np.concatenate([getattr(b, k) for b in boxes])
    with crk.Sim(crk.box_physics(b1), precision=1) as sim:
        crk.crk_load_boxes(sim.handle, [b.n for b in boxes], [crk.box_physics(b) for b in boxes],
                           cat("pos"), cat("vel"), cat("mass"), cat("u"), cat("h"), cat("species"))
        sim.n = b1.n + b2.n
        crk.crk_step_bins(sim.handle, DT_LONG, DEPTH, 1, ETA, COURANT)
        pos, vel, u = sim.state()
        bins = crk.crk_get_bins(sim.handle)
    off = 0
    for b in boxes:
        with crk.Sim(crk.box_physics(b), precision=1) as one:
            # a one-box batch: the same full sort as the two-box handle
            crk.crk_load_boxes(one.handle, [b.n], [crk.box_physics(b)], b.pos, b.vel, b.mass, b.u, b.h,
                               b.species)
            one.n = b.n
            crk.crk_step_bins(one.handle, DT_LONG, DEPTH, 1, ETA, COURANT)
            p1, v1, u1 = one.state()
            bb = crk.crk_get_bins(one.handle)
        sl = slice(off, off + b.n)
        assert np.array_equal(bins[sl], bb)
        assert np.array_equal(pos[sl], p1) and np.array_equal(vel[sl], v1) and np.array_equal(u[sl], u1)
        off += b.n


def test_bins_with_mesh_match_oracle(crk, reference):
    """Hierarchical steps with the long-range mesh: mesh half kicks around
    every long step, short-range substeps (FP64 form against the oracle)."""
    box = _box()
    op = oracle.make_params(**box.params())
    ng = 12
    ref = ob.kdk_bins(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, DT_LONG, DEPTH, 2,
                      eta=ETA, courant=COURANT, pm_grid=ng)
    with crk.Sim(crk.box_physics(box), precision=0, pm_grid=ng) as sim:
        sim.load(box)
        counts = crk.crk_step_bins(sim.handle, DT_LONG, DEPTH, 2, ETA, COURANT)
        bins = crk.crk_get_bins(sim.handle)
        pos, vel, u = sim.state()
    assert np.array_equal(counts, ref["active_counts"])
    assert np.array_equal(bins, ref["bins"])
    assert disp_err(pos, ref["pos"], box.pos, box.L) <= 1e-10
    assert rel_l2(vel, ref["vel"]) <= 1e-10
    assert rel_l2(u, ref["u"]) <= 1e-10
    # the mesh changes the outcome: it is not a no-op here
    assert rel_l2(vel, reference[1]["vel"]) > 1e-8
