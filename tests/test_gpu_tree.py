"""Direct checks of the tree (S1) and the leaf-pair lists (S2) through
crk_get_tree: every particle in exactly one leaf of one species, leaf boxes
that contain their particles, each list row free of duplicates and
symmetric, and every neighbour pair of the method's sets (hydro: gas pairs
with r < max(2h_i, 2h_j); gravity: pairs with r < r_cut) on a leaf pair of
the matching list.  The neighbour pairs come from an independent numpy
all-pairs sweep with the predicate's FP64 r^2; its per-particle counts are
checked against the oracle's first, so the pairs are the oracle's sets.
A failure names the invariant that broke, which the bit-exact set
comparisons of the parity tests cannot."""
import numpy as np
import pytest

import oracle
from paper_2510_03557_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crk():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2510_03557_gb300 import crk as c

    return c


def _pairs(pos, h, species, r_cut, L=1.0, block=512):
    """Unordered neighbour pairs (i < j) of both sets and the oracle-style
    per-particle counts (gather set r < 2h_i for gas, gravity set)."""
    N = len(pos)
    gas = species == wl.GAS
    H2 = (2.0 * h) ** 2
    hyd, grv = [], []
    gather_count = np.zeros(N, np.int64)
    grav_count = np.zeros(N, np.int64)
    for a in range(0, N, block):
        b = min(N, a + block)
        d = pos[None, :, :] - pos[a:b, None, :]      # x_j - x_i
        d = np.where(d >= 0.5 * L, d - L, d)
        d = np.where(d < -0.5 * L, d + L, d)
        r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        ii = np.arange(a, b)[:, None]
        jj = np.arange(N)[None, :]
        notself = ii != jj
        g = (r2 < r_cut * r_cut) & notself
        gath = (r2 < H2[a:b, None]) & gas[a:b, None] & gas[None, :] & notself
        union = ((r2 < H2[a:b, None]) | (r2 < H2[None, :])) & gas[a:b, None] & gas[None, :] & notself
        gather_count[a:b] = gath.sum(1)
        grav_count[a:b] = g.sum(1)
        up = jj > ii
        i1, j1 = np.nonzero(union & up)
        hyd.append(np.stack([i1 + a, j1], 1))
        i2, j2 = np.nonzero(g & up)
        grv.append(np.stack([i2 + a, j2], 1))
    return np.concatenate(hyd), np.concatenate(grv), gather_count, grav_count


def _check_tree(crk, sim, s, r_cut, cap, label):
    t = crk.crk_get_tree(sim.handle)
    N = len(s["mass"])
    order, start, count = t["order"], t["leaf_start"].astype(np.int64), t["leaf_count"].astype(np.int64)
    nl = len(start)
    # every particle in exactly one leaf
    assert np.array_equal(np.sort(order), np.arange(N)), f"{label}: order is not a permutation"
    assert nl > 0 and start[0] == 0 and count.sum() == N, f"{label}: leaves do not cover the particles"
    assert np.array_equal(start[1:], start[:-1] + count[:-1]), f"{label}: leaves overlap or leave gaps"
    assert count.min() >= 1 and count.max() <= cap, f"{label}: a leaf holds 0 or more than {cap} particles"
    leaf_of_sorted = np.repeat(np.arange(nl), count)
    leaf_of = np.empty(N, np.int64)
    leaf_of[order] = leaf_of_sorted
    # one species per leaf
    assert np.array_equal(s["species"][order], t["leaf_species"][leaf_of_sorted]), f"{label}: mixed-species leaf"
    # leaf boxes contain their particles (minimum image from the centre)
    off = s["pos"][order] - t["leaf_centre"][leaf_of_sorted]
    off = off - np.rint(off)
    over = np.abs(off) - t["leaf_half"][leaf_of_sorted].astype(np.float64)
    assert over.max() <= 0.0, f"{label}: particle {order[np.argmax(over.max(1))]} outside its leaf box"
    # rows: ascending, no duplicate, own leaf included, symmetric
    pairs = {}
    for kind in ("hydro", "grav"):
        row, col = t[kind + "_row"].astype(np.int64), t[kind + "_col"].astype(np.int64)
        assert row[0] == 0 and row[-1] == len(col) and np.all(np.diff(row) >= 0), f"{label} {kind}: bad rows"
        owner = np.repeat(np.arange(nl), np.diff(row))
        same = owner[1:] == owner[:-1]
        assert np.all(col[1:][same] > col[:-1][same]), f"{label} {kind}: row not strictly ascending"
        key = owner * nl + col
        nonempty = np.flatnonzero(np.diff(row) > 0)
        assert np.isin(nonempty * nl + nonempty, key).all(), f"{label} {kind}: a row lacks its own leaf"
        assert np.array_equal(np.sort(key), np.sort(col * nl + owner)), f"{label} {kind}: list not symmetric"
        pairs[kind] = key
        if kind == "hydro":
            gas_leaf = t["leaf_species"] == wl.GAS
            assert gas_leaf[owner].all() and gas_leaf[col].all(), f"{label}: DM leaf in the hydro list"
    # every neighbour pair of the oracle's sets lies on a listed leaf pair
    hyd, grv, gcnt, rcnt = _pairs(s["pos"], s["h"], s["species"], r_cut)
    op = oracle.make_params(box=1.0, r_cut=r_cut)
    oc, _ = oracle.neighbours(s["pos"], s["h"], s["species"], op, 0)
    og, _ = oracle.neighbours(s["pos"], s["h"], s["species"], op, 2)
    assert np.array_equal(gcnt, oc) and np.array_equal(rcnt, og), f"{label}: numpy sets differ from the oracle's"
    for kind, pr in (("hydro", hyd), ("grav", grv)):
        lk = leaf_of[pr[:, 0]] * nl + leaf_of[pr[:, 1]]
        miss = ~np.isin(lk, pairs[kind])
        assert not miss.any(), (f"{label} {kind}: {miss.sum()} neighbour pairs on unlisted leaf pairs, "
                                f"first {pr[miss][:3].tolist()}")
    return t


def _clustered_small(seed, n_gas=6000, n_dm=2000):
    rng = np.random.default_rng(seed)
    g = np.concatenate([rng.uniform(0, 1, size=(n_gas // 2, 3)),
                        (0.02 + 0.04 * rng.standard_normal((n_gas - n_gas // 2, 3))) % 1.0])
    d = np.concatenate([rng.uniform(0, 1, size=(n_dm // 2, 3)),
                        (0.6 + 0.04 * rng.standard_normal((n_dm - n_dm // 2, 3))) % 1.0])
    pos = np.concatenate([g, d])
    pos[pos >= 1.0] = 0.0
    sp = np.concatenate([np.ones(n_gas, np.uint8), np.zeros(n_dm, np.uint8)])
    perm = rng.permutation(len(sp))
    pos, sp = pos[perm], sp[perm]
    h = np.zeros(len(sp))
    h[sp == 1] = wl.knn_smoothing_lengths(pos[sp == 1], 32, 1.2)
    N = len(sp)
    return dict(pos=pos, vel=np.zeros((N, 3)), mass=np.full(N, 1.0 / N), u=np.where(sp == 1, 1.0, 0.0),
                h=h, species=sp)


@pytest.mark.parametrize("leaf_cap", [32, 64, 128])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_tree_invariants_gaussian_box(crk, precision, leaf_cap):
    box = wl.gaussian_field_box(12, seed=17)
    s = dict(pos=box.pos, vel=box.vel, mass=box.mass, u=box.u, h=box.h, species=box.species)
    with crk.Sim(crk.box_physics(box), leaf_cap=leaf_cap, precision=precision) as sim:
        sim.load(box)
        sim.forces(counts=False)
        _check_tree(crk, sim, s, box.r_cut, leaf_cap, f"gaussian cap={leaf_cap}")


@pytest.mark.parametrize("leaf_cap", [32, 128])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_tree_invariants_clustered_through_the_faces(crk, precision, leaf_cap):
    """A gas clump on the box corner (leaves across the periodic faces) and a
    DM clump inside, kNN h: variable leaf sizes and asymmetric hydro reach."""
    s = _clustered_small(seed=11)
    r_cut = 0.09
    phys = crk.physics(box=1.0, r_cut=r_cut, r_split=r_cut / 4.5, eps_soft=1e-3)
    with crk.Sim(phys, leaf_cap=leaf_cap, precision=precision) as sim:
        crk.crk_load(sim.handle, s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"])
        sim.n = len(s["mass"])
        sim.forces(counts=False)
        _check_tree(crk, sim, s, r_cut, leaf_cap, f"clustered cap={leaf_cap}")


def test_tree_invariants_after_steps_with_grown_leaves(crk):
    """Leaves kept between sorts (rebuild_every): after 3 KDK steps the
    leaves still partition the particles and their grown boxes still contain
    them; the lists still cover every neighbour pair."""
    box = wl.gaussian_field_box(12, seed=23)
    box.vel = box.vel * 30.0
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=1, rebuild_every=8) as sim:
        sim.load(box)
        sim.step(box.dt, 3)
        pos, vel, u = sim.state()
        sim.forces(counts=False)
        s = dict(pos=pos, vel=vel, mass=box.mass, u=u, h=box.h, species=box.species)
        _check_tree(crk, sim, s, box.r_cut, 64, "grown leaves")


def test_tree_needs_a_force_evaluation_first(crk):
    box = wl.gaussian_field_box(12, seed=2)
    with crk.Sim(crk.box_physics(box), precision=1) as sim:
        sim.load(box)
        with pytest.raises(crk.CrkError) as e:
            crk.crk_get_tree(sim.handle)
        assert e.value.code == crk.CRK_EINVAL
