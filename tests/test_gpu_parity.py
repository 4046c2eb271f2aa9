"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bars: neighbour-set sizes and 64-bit hashes bit-exact, over every particle;
every floating-point output within relative L2 1e-10 (FP64 plain form) or
2e-4 (FP32 mixed form) of the oracle, where relative L2 = ||gpu - oracle||_2 /
||oracle||_2 over the whole array, and, particle by particle,
|gpu_i - oracle_i| / (|oracle_i| + 1e-6 RMS(oracle)) <= 1e-8 (FP64) or 1e-2
(mixed), with |.| the Euclidean norm of the particle's row (so that one wrong
particle cannot hide inside the array's norm).
"""
import numpy as np
import pytest

import oracle
from paper_2510_03557_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-4}  # CRK_FP64, CRK_MIXED
PTOL = {0: 1e-8, 1: 1e-2}   # per particle, against |oracle_i| + 1e-6 RMS(oracle)
FLOAT_OUTPUTS = ("acc", "dudt", "rho", "A", "B", "gradA", "gradB")
ORACLE_KEY = {"acc": "acc", "dudt": "dudt", "rho": "rho", "A": "A", "B": "B", "gradA": "dA",
              "gradB": "dB"}


@pytest.fixture(scope="module")
def crk():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2510_03557_gb300 import crk as c

    return c


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def oracle_params(box_like, **kw):
    d = dict(box_like) if isinstance(box_like, dict) else box_like.params()
    d.update(kw)
    return oracle.make_params(**d)


def run_gpu(crk, s, phys, precision, leaf_cap=64, counts=True, flags=0):
    with crk.Sim(phys, leaf_cap=leaf_cap, precision=precision, flags=flags) as sim:
        crk.crk_load(sim.handle, s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"])
        sim.n = len(s["mass"])
        return sim.forces(counts=counts)


def worst_particle(a, b):
    """Largest per-particle error |a_i - b_i| / (|b_i| + 1e-6 RMS(b)), the
    norms taken over each particle's row, and that particle's position in
    the compared array."""
    a = np.asarray(a, dtype=np.float64).reshape(len(a), -1)
    b = np.asarray(b, dtype=np.float64).reshape(len(b), -1)
    if len(b) == 0:
        return 0.0, -1
    nb = np.linalg.norm(b, axis=1)
    floor = 1e-6 * np.sqrt(np.mean(nb * nb))
    den = nb + floor
    err = np.linalg.norm(a - b, axis=1) / np.where(den > 0, den, 1.0)
    k = int(np.argmax(err))
    return float(err[k]), k


def compare(out, ref, counts_ref, precision, sample=None, label="", sets_sample=None):
    """Neighbour counts and hashes over every particle (or over sets_sample
    when given), floating-point outputs over sample (every particle when
    None): relative L2 and the per-particle bound."""
    ssel = slice(None) if sets_sample is None else sets_sample
    for name, (c, h) in counts_ref.items():
        bad = np.flatnonzero(out[name + "_count"][ssel] != c[ssel])
        assert bad.size == 0, f"{label} {name} counts differ at {bad.size} particles, first {bad[:5]}"
        bad = np.flatnonzero(out[name + "_hash"][ssel] != h[ssel])
        assert bad.size == 0, f"{label} {name} hashes differ at {bad.size} particles, first {bad[:5]}"
    sel = slice(None) if sample is None else sample
    idx = np.arange(len(out["rho"]))[sel]
    tol, ptol = TOL[precision], PTOL[precision]
    for k in FLOAT_OUTPUTS:
        a, b = out[k][sel], ref[ORACLE_KEY[k]][sel]
        err = rel_l2(a, b)
        assert err <= tol, f"{label} {k}: relative L2 {err:.3e} > {tol:.1e}"
        w, at = worst_particle(a, b)
        assert w <= ptol, (f"{label} {k}: particle {idx[at]} off by {w:.3e} of its size "
                           f"(> {ptol:.0e}): gpu {np.ravel(a[at])} oracle {np.ravel(b[at])}")


def box_dict(box):
    return dict(pos=box.pos, vel=box.vel, mass=box.mass, u=box.u, h=box.h, species=box.species)


def oracle_counts(s, op):
    nc, nh = oracle.neighbours(s["pos"], s["h"], s["species"], op, 0)
    gc, gh = oracle.neighbours(s["pos"], s["h"], s["species"], op, 2)
    return {"nbr": (nc, nh), "grav": (gc, gh)}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_lattice_2x32_matches_oracle(crk, precision):
    """The 2 x 32^3 jittered lattice, every output, the whole box."""
    box = wl.jittered_lattice(32, seed=0)
    s = box_dict(box)
    op = oracle_params(box)
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op)
    assert ref["rc"] == 0
    out = run_gpu(crk, s, crk.box_physics(box), precision)
    compare(out, ref, oracle_counts(s, op), precision, label="lattice")


def _clustered(seed, n_gas=3000, n_dm=2000):
    """Half uniform, half in a Gaussian clump, species shuffled; gas h from
    the 32nd-nearest gas neighbour (as in the clustered workload), so gather
    sets are asymmetric and every m2 is well conditioned."""
    rng = np.random.default_rng(seed)
    g1 = rng.uniform(0, 1, size=(n_gas // 2, 3))
    g2 = (0.5 + 0.05 * rng.standard_normal((n_gas - n_gas // 2, 3))) % 1.0
    dm = np.concatenate([rng.uniform(0, 1, size=(n_dm // 2, 3)),
                         (0.95 + 0.05 * rng.standard_normal((n_dm - n_dm // 2, 3))) % 1.0])
    pos = np.concatenate([g1, g2, dm])
    pos[pos >= 1.0] = 0.0
    sp = np.concatenate([np.ones(n_gas, np.uint8), np.zeros(n_dm, np.uint8)])
    N = pos.shape[0]
    perm = rng.permutation(N)
    pos, sp = pos[perm], sp[perm]
    mass = np.where(sp == 1, 1.0 / n_gas, 2.0 / n_dm) * rng.uniform(0.8, 1.2, size=N)
    h = np.zeros(N)
    h[sp == 1] = wl.knn_smoothing_lengths(pos[sp == 1], 32, 1.2)
    u = np.where(sp == 1, np.exp(rng.normal(0, 0.5, size=N)), 0.0)
    vel = 0.2 * rng.standard_normal((N, 3))
    return dict(pos=pos, vel=vel, mass=mass, u=u, h=h, species=sp)


@pytest.mark.parametrize("leaf_cap", [32, 64, 128])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_clustered_variable_h_matches_oracle(crk, precision, leaf_cap):
    """Clustered gas and DM, spatially varying h, several leaves and ragged
    tails per bin, periodic wrap through the box faces."""
    s = _clustered(seed=21 + leaf_cap)
    phys = dict(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.12, r_split=0.12 / 4.5, eps_soft=1e-3)
    op = oracle.make_params(**phys)
    ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
    assert ref["rc"] == 0
    out = run_gpu(crk, s, crk.physics(**phys), precision, leaf_cap=leaf_cap)
    compare(out, ref, oracle_counts(s, op), precision, label=f"clustered cap={leaf_cap}")


@pytest.mark.parametrize("leaf_cap", [64, 128])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_force_only_path_matches_oracle(crk, precision, leaf_cap):
    """The force-only call (no neighbour-set outputs) runs the pass variants
    that skip counting and hashing; the forces are the same."""
    for s, phys in ((_clustered(seed=77),
                     dict(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.12, r_split=0.12 / 4.5, eps_soft=1e-3)),
                    (box_dict(wl.jittered_lattice(20, seed=8)), wl.jittered_lattice(20, seed=8).params())):
        op = oracle.make_params(**phys)
        ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
        assert ref["rc"] == 0
        out = run_gpu(crk, s, crk.physics(**phys), precision, leaf_cap=leaf_cap, counts=False)
        compare(out, ref, {}, precision, label=f"force-only cap={leaf_cap}")


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_momentum_and_energy_rates_vanish(crk, precision):
    """Pairwise antisymmetry: sum m a = 0 with gravity; without gravity the
    hydro rates also conserve energy, sum m (v . a + du/dt) = 0 (the energy
    rate the library reports), both to roundoff of the form's arithmetic."""
    s = _clustered(seed=5)
    phys = dict(box=1.0, r_cut=0.12, r_split=0.12 / 4.5, eps_soft=1e-3)
    out = run_gpu(crk, s, crk.physics(**phys), precision, counts=False)
    ma = s["mass"][:, None] * out["acc"]
    scale = np.abs(ma).sum()
    rel = np.abs(out["momentum_rate"]).max() / scale
    assert rel < (1e-13 if precision == 0 else 1e-5)
    # the library's FP64 sum agrees with the host sum of its own outputs
    assert np.allclose(out["momentum_rate"], ma.sum(0), rtol=0, atol=1e-9 * scale)
    # hydro alone (G = 0): the energy rate vanishes and equals the host sum
    out = run_gpu(crk, s, crk.physics(**dict(phys, G=0.0)), precision, counts=False)
    terms = s["mass"] * (np.einsum("ij,ij->i", s["vel"], out["acc"]) + out["dudt"])
    escale = np.abs(s["mass"] * np.einsum("ij,ij->i", s["vel"], out["acc"])).sum() + \
        np.abs(s["mass"] * out["dudt"]).sum()
    assert escale > 0
    assert abs(out["energy_rate"]) / escale < (1e-13 if precision == 0 else 1e-5)
    assert abs(out["energy_rate"] - terms.sum()) <= 1e-9 * escale
    pscale = np.abs(s["mass"][:, None] * out["acc"]).sum()
    assert np.abs(out["momentum_rate"]).max() / pscale < (1e-13 if precision == 0 else 1e-5)


def test_full_size_gaussian_field_sampled(crk):
    """2 x 128^3, mixed form: the neighbour sets of all 4.19 M particles
    bit-exact, the forces of sampled particles checked one by one against
    the oracle."""
    box = wl.gaussian_field_box(128, seed=1)
    s = box_dict(box)
    op = oracle_params(box)
    out = run_gpu(crk, s, crk.box_physics(box), 1)
    rng = np.random.default_rng(0)
    gas = np.nonzero(box.species == wl.GAS)[0]
    dm = np.nonzero(box.species == wl.DM)[0]
    sample = np.sort(np.concatenate([rng.choice(gas, 48, replace=False), rng.choice(dm, 16, replace=False)]))
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, sample=sample)
    assert ref["rc"] == 0
    nc, nh = oracle.neighbours(box.pos, box.h, box.species, op, 0)
    gc, gh = oracle.neighbours(box.pos, box.h, box.species, op, 2)
    compare(out, ref, {"nbr": (nc, nh), "grav": (gc, gh)}, 1, sample=sample, label="2x128^3")
    assert len(nc) == box.n and len(gc) == box.n   # the sets were compared over every particle
    # every particle has a full neighbourhood (~270 for gas, paper Sec. IV-B1)
    assert 200 < out["nbr_count"][gas].mean() < 330


_CLUSTERED_CACHE = {}


def _clustered_2x64(nsphere):
    """The clustered generator at 2 x 64^3 with its oracle neighbour sets,
    computed once per sphere count for both forms."""
    if nsphere not in _CLUSTERED_CACHE:
        box = wl.clustered_box(64, seed=3, nsphere=nsphere)
        op = oracle_params(box)
        sets = {"nbr": oracle.neighbours(box.pos, box.h, box.species, op, 0),
                "grav": oracle.neighbours(box.pos, box.h, box.species, op, 2)}
        gas = np.flatnonzero(box.species == wl.GAS)
        rng = np.random.default_rng(64 + nsphere)
        dense = gas[np.argsort(box.h[gas], kind="stable")[:64]]      # smallest h: densest gas
        rest = np.setdiff1d(np.arange(box.n), dense)
        sample = np.sort(np.concatenate([dense, rng.choice(rest, 192, replace=False)]))
        ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, sample=sample)
        assert ref["rc"] == 0
        _CLUSTERED_CACHE[nsphere] = (box, sets, sample, ref)
    return _CLUSTERED_CACHE[nsphere]


@pytest.mark.parametrize("nsphere", [512, 8], ids=["512-spheres", "8-dense-cores"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_clustered_2x64_matches_oracle(crk, precision, nsphere):
    """The clustered workload's generator (half uniform, half in Plummer
    spheres of scale 0.002, kNN h) at 2 x 64^3 = 524,288 particles: the
    neighbour sets of every particle bit-exact, and 256 sampled particles,
    the 64 densest gas particles among them, checked one by one.  With 8
    spheres each core holds 32,768 particles, as each of the 512 cores of the
    2 x 256^3 box does, so core particles see tens of thousands of gravity
    neighbours and hundreds of hydro neighbours, as at full size."""
    box, sets, sample, ref = _clustered_2x64(nsphere)
    out = run_gpu(crk, box_dict(box), crk.box_physics(box), precision, leaf_cap=128)
    compare(out, ref, sets, precision, sample=sample, label=f"clustered 2x64^3 nsphere={nsphere}")
    if nsphere == 8:
        assert sets["grav"][0].max() > 20000     # the dense cores are really reached
    if precision == 1:
        # the mixed form with gravity pairs evaluated once, the partial sums
        # added by atomics (a force-only evaluation: counted ones gather)
        once = run_gpu(crk, box_dict(box), crk.box_physics(box), 1, leaf_cap=128, counts=False,
                       flags=crk.CRK_FLAG_GRAVITY_PAIRS_ONCE)
        compare(once, ref, {}, 1, sample=sample, label=f"clustered 2x64^3 nsphere={nsphere}, pairs once")
        assert rel_l2(once["acc"], out["acc"]) <= TOL[1]
        # and the hydro rates with each union pair evaluated once as well
        both = run_gpu(crk, box_dict(box), crk.box_physics(box), 1, leaf_cap=128, counts=False,
                       flags=crk.CRK_FLAG_GRAVITY_PAIRS_ONCE | crk.CRK_FLAG_HYDRO_PAIRS_ONCE)
        compare(both, ref, {}, 1, sample=sample, label=f"clustered 2x64^3 nsphere={nsphere}, both once")
        assert rel_l2(both["dudt"], out["dudt"]) <= TOL[1]


@pytest.mark.parametrize("leaf_cap", [32, 64, 128])
def test_gravity_pairs_once_matches_the_gather_form(crk, leaf_cap):
    """Mixed form: gravity with each unordered pair evaluated once (atomics)
    against the default gather form and the oracle on the clustered inputs
    with periodic wraps; the gather form gives bit-identical repeated
    evaluations, the pairs-once form agrees with it to rounding and keeps the
    total momentum rate at roundoff."""
    s = _clustered(seed=91)
    phys = dict(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.12, r_split=0.12 / 4.5, eps_soft=1e-3)
    op = oracle.make_params(**phys)
    ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
    assert ref["rc"] == 0
    d1 = run_gpu(crk, s, crk.physics(**phys), 1, leaf_cap=leaf_cap, counts=False)
    d2 = run_gpu(crk, s, crk.physics(**phys), 1, leaf_cap=leaf_cap, counts=False)
    assert np.array_equal(d1["acc"], d2["acc"])
    once = run_gpu(crk, s, crk.physics(**phys), 1, leaf_cap=leaf_cap, counts=False,
                   flags=crk.CRK_FLAG_GRAVITY_PAIRS_ONCE)
    compare(once, ref, {}, 1, label=f"pairs once cap={leaf_cap}")
    assert rel_l2(once["acc"], d1["acc"]) <= 1e-5
    ma = s["mass"][:, None] * once["acc"]
    assert np.abs(once["momentum_rate"]).max() / np.abs(ma).sum() < 1e-5


@pytest.mark.parametrize("leaf_cap", [32, 64, 128])
def test_hydro_pairs_once_matches_the_gather_form(crk, leaf_cap):
    """Mixed form: the hydro rates with each union pair evaluated once by its
    lower-indexed particle (the partner's side, -F_ij / m_j and the same
    energy term, added by an atomic) against the gather form and the oracle
    on the clustered inputs with periodic wraps.  The pairwise antisymmetry
    keeps the total hydro momentum rate at roundoff and the energy rate of
    the G = 0 box at the oracle's."""
    s = _clustered(seed=93)
    phys = dict(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.12, r_split=0.12 / 4.5, eps_soft=1e-3)
    op = oracle.make_params(**phys)
    ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
    assert ref["rc"] == 0
    gat = run_gpu(crk, s, crk.physics(**phys), 1, leaf_cap=leaf_cap, counts=True)
    once = run_gpu(crk, s, crk.physics(**phys), 1, leaf_cap=leaf_cap, counts=True,
                   flags=crk.CRK_FLAG_HYDRO_PAIRS_ONCE)
    compare(once, ref, oracle_counts(s, op), 1, label=f"hydro pairs once cap={leaf_cap}")
    assert rel_l2(once["dudt"], gat["dudt"]) <= 1e-5 and rel_l2(once["acc"], gat["acc"]) <= 1e-5
    # G = 0: only hydro moves the particles, so the total momentum rate is the
    # hydro pass's alone
    phys0 = dict(phys, G=0.0)
    h0 = run_gpu(crk, s, crk.physics(**phys0), 1, leaf_cap=leaf_cap, counts=False,
                 flags=crk.CRK_FLAG_HYDRO_PAIRS_ONCE)
    ma = s["mass"][:, None] * h0["acc"]
    assert np.abs(ma.sum(0)).max() / np.abs(ma).sum() < 1e-5


def _clustered_smooth_h(seed, n_gas=2500, n_dm=1500, h0=0.09):
    """Half uniform, half in a Gaussian clump, species shuffled, gas h from a
    smooth field h0 + 0.04 sin(5x) cos(3y).  With h0 = 0.09 the uniform
    half's smallest supports hold only a few neighbours, and some gas
    particle's second-moment matrix is singular."""
    rng = np.random.default_rng(seed)
    g1 = rng.uniform(0, 1, size=(n_gas // 2, 3))
    g2 = (0.5 + 0.05 * rng.standard_normal((n_gas - n_gas // 2, 3))) % 1.0
    dm = np.concatenate([rng.uniform(0, 1, size=(n_dm // 2, 3)),
                         (0.3 + 0.05 * rng.standard_normal((n_dm - n_dm // 2, 3))) % 1.0])
    pos = np.concatenate([g1, g2, dm])
    pos[pos >= 1.0] = 0.0
    sp = np.concatenate([np.ones(n_gas, np.uint8), np.zeros(n_dm, np.uint8)])
    N = pos.shape[0]
    perm = rng.permutation(N)
    pos, sp = pos[perm], sp[perm]
    mass = np.where(sp == 1, 1.0 / n_gas, 2.0 / n_dm) * rng.uniform(0.8, 1.2, size=N)
    h = np.where(sp == 1, h0 + 0.04 * np.sin(5.0 * pos[:, 0]) * np.cos(3.0 * pos[:, 1]), 0.0)
    u = np.where(sp == 1, np.exp(rng.normal(0, 0.5, size=N)), 0.0)
    vel = 0.2 * rng.standard_normal((N, 3))
    return dict(pos=pos, vel=vel, mass=mass, u=u, h=h, species=sp)


@pytest.mark.parametrize("seed", [53, 149])
@pytest.mark.parametrize("leaf_cap", [32, 128])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_smooth_field_h_singular_inputs_are_reported(crk, precision, leaf_cap, seed):
    """The smooth-h inputs with h0 = 0.09 leave gas particles in the uniform
    half with no or one neighbour, whose m2 is singular: the oracle reports
    CRK_ESINGULAR, and so does each GPU form (never a NaN result)."""
    s = _clustered_smooth_h(seed=seed)
    phys = dict(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.12, r_split=0.12 / 4.5, eps_soft=1e-3)
    op = oracle.make_params(**phys)
    ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
    assert ref["rc"] == crk.CRK_ESINGULAR
    with pytest.raises(crk.CrkError) as e:
        run_gpu(crk, s, crk.physics(**phys), precision, leaf_cap=leaf_cap)
    assert e.value.code == crk.CRK_ESINGULAR


@pytest.mark.parametrize("leaf_cap", [32, 64, 128])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_smooth_field_h_matches_oracle(crk, precision, leaf_cap):
    """Smoothly varying h (not kNN h), raised to h0 = 0.12 so every m2 is
    invertible: gather sets from about twenty neighbours in the uniform half
    to about a thousand in the clump."""
    s = _clustered_smooth_h(seed=21 + leaf_cap, h0=0.12)
    phys = dict(box=1.0, G=1.0, gamma=5.0 / 3.0, r_cut=0.12, r_split=0.12 / 4.5, eps_soft=1e-3)
    op = oracle.make_params(**phys)
    ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
    assert ref["rc"] == 0
    out = run_gpu(crk, s, crk.physics(**phys), precision, leaf_cap=leaf_cap)
    compare(out, ref, oracle_counts(s, op), precision, label=f"smooth h cap={leaf_cap}")


# ------------------------------------------------------------- edge cases
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_fewer_particles_than_one_leaf_and_box_faces(crk, precision):
    rng = np.random.default_rng(3)
    N = 23
    pos = 0.05 * rng.standard_normal((N, 3))      # a clump around the box corner
    pos[0] = [0.0, 0.0, 0.0]
    pos[1] = [np.nextafter(1.0, 0.0), 0.0, np.nextafter(1.0, 0.0)]
    pos[2] = [0.0, np.nextafter(1.0, 0.0), 0.02]
    pos = np.mod(pos, 1.0)
    pos[pos >= 1.0] = 0.0
    sp = np.array([1] * 15 + [0] * 8, np.uint8)
    s = dict(pos=pos, vel=0.1 * rng.standard_normal((N, 3)), mass=np.full(N, 1.0 / N),
             u=np.where(sp == 1, 1.0, 0.0), h=np.where(sp == 1, 0.12, 0.0), species=sp)
    phys = dict(box=1.0, r_cut=0.3, r_split=0.3 / 4.5, eps_soft=1e-3)
    op = oracle.make_params(**phys)
    ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
    assert ref["rc"] == 0
    out = run_gpu(crk, s, crk.physics(**phys), precision, leaf_cap=32)
    compare(out, ref, oracle_counts(s, op), precision, label="tiny")


@pytest.mark.parametrize("only", [0, 1], ids=["all-dm", "all-gas"])
def test_single_species(crk, only):
    box = wl.jittered_lattice(10, seed=4)
    keep = box.species == only
    s = {k: v[keep] for k, v in box_dict(box).items()}
    op = oracle_params(box)
    ref = oracle.forces(s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"], op)
    for precision in (0, 1):
        out = run_gpu(crk, s, crk.box_physics(box), precision)
        compare(out, ref, oracle_counts(s, op), precision, label=f"species={only}")


def test_empty_input(crk):
    with crk.Sim(crk.physics()) as sim:
        z = np.zeros((0, 3))
        crk.crk_load(sim.handle, z, z, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0, np.uint8))
        sim.n = 0
        out = sim.forces()
        assert out["acc"].shape == (0, 3)
        sim.step(1e-3, 2)


def test_all_gas_at_one_point_reports_singular(crk):
    N = 40
    s = dict(pos=np.full((N, 3), 0.5), vel=np.zeros((N, 3)), mass=np.full(N, 1.0 / N),
             u=np.ones(N), h=np.full(N, 0.05), species=np.ones(N, np.uint8))
    for precision in (0, 1):
        with pytest.raises(crk.CrkError) as e:
            run_gpu(crk, s, crk.physics(r_cut=0.1), precision)
        assert e.value.code == crk.CRK_ESINGULAR


def test_invalid_inputs_are_rejected(crk):
    N = 10
    base = dict(pos=np.full((N, 3), 0.25), vel=np.zeros((N, 3)), mass=np.full(N, 0.1),
                u=np.ones(N), h=np.full(N, 0.05), species=np.ones(N, np.uint8))
    bad_pos = dict(base, pos=base["pos"].copy())
    bad_pos["pos"][3, 1] = 1.0                      # must be < L
    bad_h = dict(base, h=np.full(N, 0.3))           # 2h >= L/2
    bad_m = dict(base, mass=np.full(N, -1.0))
    for s in (bad_pos, bad_h, bad_m):
        with crk.Sim(crk.physics(r_cut=0.1)) as sim:
            with pytest.raises(crk.CrkError) as e:
                crk.crk_load(sim.handle, s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"])
            assert e.value.code == crk.CRK_EINVAL
    with pytest.raises(crk.CrkError):
        crk.crk_create(crk.params(leaf_cap=48))
    with pytest.raises(crk.CrkError):
        crk.Sim(crk.physics(r_cut=0.6)).load(wl.jittered_lattice(4))


# ------------------------------------------------------------------ KDK
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_kdk_steps_match_oracle(crk, precision):
    box = wl.gaussian_field_box(16, seed=7)
    box.vel = box.vel * 20.0
    op = oracle_params(box)
    nsteps, dt = 3, 1e-3
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, dt, nsteps)
    with crk.Sim(crk.box_physics(box), precision=precision) as sim:
        sim.load(box)
        sim.step(dt, nsteps)
        pos, vel, u = sim.state()
        mom, energy, nfloor = crk.crk_get_sums(sim.handle)
    d = pos - ref["pos"]
    d = np.where(d > 0.5, d - 1.0, d)
    d = np.where(d < -0.5, d + 1.0, d)
    tol = TOL[precision]
    disp = np.linalg.norm(ref["pos"] - box.pos) + 1e-300
    assert np.linalg.norm(d) / disp <= tol
    assert rel_l2(vel, ref["vel"]) <= tol
    assert rel_l2(u, ref["u"]) <= tol
    m = box.mass
    p0 = (m[:, None] * box.vel).sum(0)
    assert np.max(np.abs(np.array(mom) - p0)) <= 1e-6 * np.abs(m[:, None] * box.vel).sum()


# ---------------------------------------------------------------- batched
def _global_hash(box, offset, kind):
    """Neighbour-set hash with ids offset by the box's position in the
    batched load (independent numpy all-pairs sets, same predicate)."""
    pos, h, sp = box.pos, box.h, box.species
    d = pos[None, :, :] - pos[:, None, :]
    d = np.where(d >= 0.5, d - 1.0, d)
    d = np.where(d < -0.5, d + 1.0, d)
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    eye = np.eye(box.n, dtype=bool)
    if kind == 0:
        gas = sp == wl.GAS
        m = (r2 < ((2.0 * h) ** 2)[:, None]) & gas[:, None] & gas[None, :] & ~eye
    else:
        m = (r2 < box.r_cut * box.r_cut) & ~eye
    ids = wl.splitmix64(np.arange(box.n, dtype=np.uint64) + np.uint64(offset))
    with np.errstate(over="ignore"):
        return np.array([np.sum(ids[row], dtype=np.uint64) for row in m], dtype=np.uint64)


def test_batched_boxes_match_each_box_alone(crk):
    boxes = [wl.gaussian_field_box(n, seed=100 + n) for n in (10, 12, 16)]
    cat = wl.concat_boxes(boxes)
    phys = [crk.box_physics(b) for b in boxes]
    for precision in (0, 1):
        with crk.Sim(phys[0], precision=precision) as sim:
            crk.crk_load_boxes(sim.handle, [b.n for b in boxes], phys, cat["pos"], cat["vel"],
                               cat["mass"], cat["u"], cat["h"], cat["species"])
            sim.n = int(cat["offsets"][-1])
            out = sim.forces()
        for b, box in enumerate(boxes):
            lo, hi = cat["offsets"][b], cat["offsets"][b + 1]
            part = {k: (v[lo:hi] if isinstance(v, np.ndarray) and v.shape[:1] == (sim.n,) else v)
                    for k, v in out.items()}
            op = oracle_params(box)
            ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op)
            # hashes of a batched load are over the global (load-order) index
            counts = {}
            for name, kind in (("nbr", 0), ("grav", 2)):
                c, _ = oracle.neighbours(box.pos, box.h, box.species, op, kind)
                counts[name] = (c, _global_hash(box, lo, kind))
            compare(part, ref, counts, precision, label=f"box {b}")


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_leaves_kept_between_rebuilds_match_the_oracle(crk, precision):
    """Sorting into leaves every 4th step only (the boxes grow in between):
    6 KDK steps match the oracle's KDK; and a force evaluation on leaves
    built 3 steps earlier gives the oracle's neighbour sets."""
    box = wl.gaussian_field_box(16, seed=31)
    op = oracle_params(box)
    steps = 6
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, op, box.dt, steps)
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=precision, rebuild_every=4) as sim:
        sim.load(box)
        sim.step(box.dt, steps)
        pos, vel, u = sim.state()
    tol = TOL[precision]
    assert rel_l2(vel, ref["vel"]) <= tol
    assert rel_l2(u, ref["u"]) <= tol
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=precision, rebuild_every=10) as sim:
        sim.load(box)
        sim.step(box.dt, 3)
        out = sim.forces(counts=True)  # leaves of the initial evaluation, boxes grown
        pos, vel, u = sim.state()
    moved = box_dict(box)
    moved.update(pos=pos, vel=vel, u=u)
    cref = oracle_counts(moved, op)
    for name in ("nbr", "grav"):
        assert np.array_equal(out[name + "_count"], cref[name][0]), name
        assert np.array_equal(out[name + "_hash"], cref[name][1]), name


def test_autotune_over_capacity_and_pair_decomposition(crk):
    """The two-axis autotuner times every (capacity, decomposition) pair --
    the decomposition a bit set of gravity pairs-once and hydro pairs-once --
    keeps the fastest, and the forces of the chosen configuration equal the
    oracle's."""
    box = wl.gaussian_field_box(16, seed=22)
    op = oracle_params(box)
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op)
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=1) as sim:
        sim.load(box)
        cap, form, grid = crk.crk_autotune_ex(sim.handle, (32, 128))
        assert set(grid) == {(c, f) for c in (32, 128) for f in range(4)}
        assert all(v > 0 for v in grid.values()) and grid[(cap, form)] == min(grid.values())
        out = sim.forces(counts=False)
        compare(out, ref, {}, 1, label=f"autotuned cap={cap} form={form}")
        with pytest.raises(crk.CrkError) as e:
            crk.crk_autotune_ex(sim.handle, (64,), (4,))
        assert e.value.code == crk.CRK_EINVAL


def test_autotune_keeps_the_fastest_capacity_and_the_forces(crk):
    box = wl.gaussian_field_box(16, seed=21)
    op = oracle_params(box)
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op)
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=1) as sim:
        sim.load(box)
        best, ms = crk.crk_autotune(sim.handle, (32, 64, 128))
        assert best in (32, 64, 128) and set(ms) == {32, 64, 128}
        assert all(v > 0 for v in ms.values()) and ms[best] == min(ms.values())
        out = sim.forces(counts=True)
        compare(out, ref, oracle_counts(box_dict(box), op), 1, label=f"autotuned cap={best}")
        with pytest.raises(crk.CrkError) as e:
            crk.crk_autotune(sim.handle, (48,))
        assert e.value.code == crk.CRK_EINVAL


def test_batched_step_matches_single_box_steps(crk):
    boxes = [wl.gaussian_field_box(n, seed=200 + n) for n in (10, 16)]
    cat = wl.concat_boxes(boxes)
    phys = [crk.box_physics(b) for b in boxes]
    dts = [1e-3, 2e-3]
    with crk.Sim(phys[0], precision=0) as sim:
        crk.crk_load_boxes(sim.handle, [b.n for b in boxes], phys, cat["pos"], cat["vel"],
                           cat["mass"], cat["u"], cat["h"], cat["species"])
        crk.crk_step_boxes(sim.handle, dts, 2)
        n = int(cat["offsets"][-1])
        pos, vel, u = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
        crk.crk_get_state(sim.handle, pos, vel, u)
    for b, box in enumerate(boxes):
        lo, hi = cat["offsets"][b], cat["offsets"][b + 1]
        ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, oracle_params(box),
                         dts[b], 2)
        assert rel_l2(vel[lo:hi], ref["vel"]) <= 1e-10
        assert rel_l2(u[lo:hi], ref["u"]) <= 1e-10


# ---------------------------------------------------------------- service
def _job_boxes():
    return [wl.gaussian_field_box(n, seed=300 + i) for i, n in enumerate((10, 12, 10, 16, 11))]


def _run_service(crk, boxes, nsteps, precision=1, max_slots=8):
    svc = crk.crk_service_create(8 << 30, max_slots, precision=precision)
    try:
        tickets = [crk.crk_submit(svc, crk.box_physics(b), b.pos, b.vel, b.mass, b.u, b.h,
                                  b.species, 1e-3, nsteps) for b in boxes]
        return [crk.crk_poll(svc, t, b.n, -1) for t, b in zip(tickets, boxes)]
    finally:
        crk.crk_service_destroy(svc)


def test_service_result_is_the_same_alone_and_in_the_mix(crk):
    boxes = _job_boxes()
    mixed = _run_service(crk, boxes, 4)
    for i in (0, 3):
        alone = _run_service(crk, [boxes[i]], 4)[0]
        # boxes never interact and every per-leaf sum runs in a fixed order
        assert np.array_equal(alone["pos"], mixed[i]["pos"])
        assert np.array_equal(alone["vel"], mixed[i]["vel"])
        assert np.array_equal(alone["u"], mixed[i]["u"])


def test_service_size_classes_give_the_results_of_one_class(crk):
    """Jobs of two size classes (below and above 65,536 particles) run in
    separate lanes side by side; each result equals the same job run with a
    single class and the job run alone, bit for bit."""
    boxes = [wl.gaussian_field_box(10, seed=610), wl.gaussian_field_box(34, seed=634),
             wl.gaussian_field_box(12, seed=612)]
    assert boxes[1].n >= 65536 > boxes[0].n
    svc = crk.crk_service_create(8 << 30, 4, size_classes=1)
    try:
        ts = [crk.crk_submit(svc, crk.box_physics(b), b.pos, b.vel, b.mass, b.u, b.h, b.species,
                             1e-3, 3) for b in boxes]
        one = [crk.crk_poll(svc, t, b.n, -1) for t, b in zip(ts, boxes)]
    finally:
        crk.crk_service_destroy(svc)
    lanes = _run_service(crk, boxes, 3)
    for b, x, y in zip(boxes, lanes, one):
        alone = _run_service(crk, [b], 3)[0]
        for k in ("pos", "vel", "u"):
            assert np.array_equal(x[k], y[k]) and np.array_equal(x[k], alone[k]), (b.n, k)


def test_service_reuses_freed_slots(crk):
    """Two slots, six jobs of different sizes and lengths: every freed slot
    takes the next job while the removed job's particles still sit in the
    arrays until the next sort.  Each result equals the job run alone."""
    jobs = [(wl.gaussian_field_box(n, seed=400 + k), steps)
            for k, (n, steps) in enumerate(((16, 2), (10, 5), (12, 1), (14, 3), (11, 2), (10, 1)))]
    svc = crk.crk_service_create(8 << 30, 2)
    try:
        tickets = [crk.crk_submit(svc, crk.box_physics(b), b.pos, b.vel, b.mass, b.u, b.h,
                                  b.species, 1e-3, steps) for b, steps in jobs]
        mixed = [crk.crk_poll(svc, t, b.n, -1) for t, (b, _) in zip(tickets, jobs)]
    finally:
        crk.crk_service_destroy(svc)
    for (b, steps), r in zip(jobs, mixed):
        alone = _run_service(crk, [b], steps)[0]
        assert np.array_equal(alone["pos"], r["pos"])
        assert np.array_equal(alone["vel"], r["vel"])
        assert np.array_equal(alone["u"], r["u"])


def test_service_resumes_a_cancelled_job_from_its_snapshot_bit_exactly(crk):
    """Checkpoint/resume: a job's service is cancelled mid-run (the host-side
    failure); the job resubmitted to a new service from its last snapshot
    ends exactly where the run without interruption ends."""
    import time

    box = wl.gaussian_field_box(12, seed=501)
    steps = 60
    ref = _run_service(crk, [box], steps)[0]
    svc = crk.crk_service_create(8 << 30, 4, snapshot_every=5)
    try:
        t = crk.crk_submit(svc, crk.box_physics(box), box.pos, box.vel, box.mass, box.u, box.h,
                           box.species, box.dt, steps)
        snap = None
        deadline = time.time() + 60
        while time.time() < deadline:
            snap = crk.crk_service_snapshot(svc, t, box.n)
            if snap is not None and snap["steps_done"] >= 10:
                break
            time.sleep(1e-3)
        assert snap is not None and snap["steps_done"] % 5 == 0 and 10 <= snap["steps_done"] <= steps
        crk.crk_service_cancel(svc)
        try:
            crk.crk_poll(svc, t, box.n, -1)   # finished just before the cancel, or cancelled
        except crk.CrkError as e:
            assert e.code == crk.CRK_ECANCELED
    finally:
        crk.crk_service_destroy(svc)
    svc2 = crk.crk_service_create(8 << 30, 4)
    try:
        t2 = crk.crk_submit(svc2, crk.box_physics(box), snap["pos"], snap["vel"], box.mass, snap["u"],
                            box.h, box.species, box.dt, steps, resume=snap)
        res = crk.crk_poll(svc2, t2, box.n, -1)
    finally:
        crk.crk_service_destroy(svc2)
    assert np.array_equal(res["pos"], ref["pos"])
    assert np.array_equal(res["vel"], ref["vel"])
    assert np.array_equal(res["u"], ref["u"])


def test_service_resumed_fp64_job_matches_oracle(crk):
    """Checkpoint/resume against the oracle: an FP64 job snapshotted every 4
    steps, its service cancelled after a snapshot, the job resubmitted from
    that snapshot; its final state equals the oracle's uninterrupted KDK over
    all its steps."""
    import time

    box = wl.gaussian_field_box(12, seed=503)
    box.vel = box.vel * 10.0
    steps = 16
    svc = crk.crk_service_create(8 << 30, 4, precision=0, snapshot_every=4)
    try:
        t = crk.crk_submit(svc, crk.box_physics(box), box.pos, box.vel, box.mass, box.u, box.h,
                           box.species, box.dt, steps)
        snap = None
        deadline = time.time() + 60
        while time.time() < deadline:
            snap = crk.crk_service_snapshot(svc, t, box.n)
            if snap is not None and snap["steps_done"] >= 4:
                break
            time.sleep(1e-4)
        assert snap is not None and snap["steps_done"] % 4 == 0 and 4 <= snap["steps_done"] <= steps
        crk.crk_service_cancel(svc)
        try:
            crk.crk_poll(svc, t, box.n, -1)
        except crk.CrkError as e:
            assert e.code == crk.CRK_ECANCELED
    finally:
        crk.crk_service_destroy(svc)
    svc2 = crk.crk_service_create(8 << 30, 4, precision=0)
    try:
        t2 = crk.crk_submit(svc2, crk.box_physics(box), snap["pos"], snap["vel"], box.mass, snap["u"],
                            box.h, box.species, box.dt, steps, resume=snap)
        res = crk.crk_poll(svc2, t2, box.n, -1)
    finally:
        crk.crk_service_destroy(svc2)
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, oracle_params(box), box.dt, steps)
    d = (res["pos"] - ref["pos"] + 0.5) % 1.0 - 0.5
    disp = np.linalg.norm((ref["pos"] - box.pos + 0.5) % 1.0 - 0.5)
    assert np.linalg.norm(d) / disp <= 1e-10
    assert rel_l2(res["vel"], ref["vel"]) <= 1e-10
    assert rel_l2(res["u"], ref["u"]) <= 1e-10
    w, _ = worst_particle(res["vel"], ref["vel"])
    assert w <= PTOL[0]


def test_service_matches_oracle(crk):
    boxes = _job_boxes()[:3]
    res = _run_service(crk, boxes, 3, precision=0)
    for b, r in zip(boxes, res):
        ref = oracle.kdk(b.pos, b.vel, b.mass, b.u, b.h, b.species, oracle_params(b), 1e-3, 3)
        assert rel_l2(r["vel"], ref["vel"]) <= 1e-10
        assert rel_l2(r["u"], ref["u"]) <= 1e-10
        assert r["latency_ns"] > 0


def test_service_admission_refuses_a_job_over_budget(crk):
    svc = crk.crk_service_create(1 << 20, 4)
    try:
        b = wl.gaussian_field_box(16, seed=1)
        with pytest.raises(crk.CrkError) as e:
            crk.crk_submit(svc, crk.box_physics(b), b.pos, b.vel, b.mass, b.u, b.h, b.species, 1e-3, 1)
        assert e.value.code == crk.CRK_EINVAL
        with pytest.raises(crk.CrkError) as e:
            crk.crk_poll(svc, 12345, 1, 0)
        assert e.value.code == crk.CRK_ENOTFOUND
    finally:
        crk.crk_service_destroy(svc)


def test_service_reports_a_bad_job_and_keeps_serving(crk):
    boxes = _job_boxes()[:2]
    bad = wl.gaussian_field_box(10, seed=9)
    bad.pos = bad.pos.copy()
    bad.pos[0, 0] = 2.0
    svc = crk.crk_service_create(8 << 30, 4)
    try:
        t_bad = crk.crk_submit(svc, crk.box_physics(bad), bad.pos, bad.vel, bad.mass, bad.u, bad.h,
                               bad.species, 1e-3, 2)
        ts = [crk.crk_submit(svc, crk.box_physics(b), b.pos, b.vel, b.mass, b.u, b.h, b.species,
                             1e-3, 2) for b in boxes]
        with pytest.raises(crk.CrkError) as e:
            crk.crk_poll(svc, t_bad, bad.n, -1)
        assert e.value.code == crk.CRK_EINVAL
        for t, b in zip(ts, boxes):
            assert crk.crk_poll(svc, t, b.n, -1) is not None
    finally:
        crk.crk_service_destroy(svc)


# ------------------------------------------------------------------ friends-of-friends
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_fof_groups_equal_the_oracle(crk, precision):
    """Group labels (smallest original index per group) and counts are
    integers: bit-exact against the oracle, for DM only and all species, at
    the usual b = 0.2 mean spacings and near percolation."""
    box = wl.clustered_box(24, seed=41, knn=False)
    phys = box.params()
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=precision) as sim:
        sim.load(box)
        for b_over, mask in ((0.2, 1), (0.2, 3), (0.75, 1)):
            b = b_over / 24
            assert b <= phys["r_cut"]
            grp, ng = crk.crk_fof(sim.handle, b, mask)
            ref, ref_ng = oracle.fof(box.pos, box.species, phys["box"], b, mask)
            assert ng == ref_ng, (b_over, mask)
            assert np.array_equal(grp, ref), (b_over, mask)
            assert ng < np.count_nonzero(ref >= 0)  # groups really formed
        with pytest.raises(crk.CrkError) as e:
            crk.crk_fof(sim.handle, 2 * phys["r_cut"], 1)
        assert e.value.code == crk.CRK_EINVAL


def test_fof_groups_stay_inside_their_box(crk):
    boxes = [wl.clustered_box(n, seed=60 + n, knn=False) for n in (16, 20)]
    cat = wl.concat_boxes(boxes)
    phys = [crk.box_physics(b) for b in boxes]
    b = 0.2 / 20
    with crk.Sim(phys[0], precision=1) as sim:
        crk.crk_load_boxes(sim.handle, [x.n for x in boxes], phys, cat["pos"], cat["vel"], cat["mass"],
                           cat["u"], cat["h"], cat["species"])
        sim.n = int(cat["offsets"][-1])
        grp, ng = crk.crk_fof(sim.handle, b, 1)
    total = 0
    for k, bx in enumerate(boxes):
        lo, hi = cat["offsets"][k], cat["offsets"][k + 1]
        ref, ref_ng = oracle.fof(bx.pos, bx.species, bx.params()["box"], b, 1)
        ref = np.where(ref >= 0, ref + lo, -1)
        assert np.array_equal(grp[lo:hi], ref)
        total += ref_ng
    assert ng == total


# ------------------------------------------- list sizes from the last step
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_lists_sized_from_last_step_equal_counted_lists(crk, precision):
    """The second force evaluation sizes its hydro lists from the first one's
    counts (no count pass): the outputs are bit-identical."""
    box = wl.gaussian_field_box(16, seed=3)
    with crk.Sim(crk.box_physics(box), precision=precision) as sim:
        sim.load(box)
        a = sim.forces(counts=True)
        b = sim.forces(counts=True)
    for k in FLOAT_OUTPUTS + ("nbr_count", "nbr_hash", "grav_count", "grav_hash"):
        assert np.array_equal(a[k], b[k]), k


def test_lists_that_outgrow_last_step_sizes_are_counted_again(crk):
    """Compress the box after a step so every list grows far beyond the
    margin: the fill pass asks for a count pass and the forces still equal
    the oracle's at the new positions."""
    box = wl.jittered_lattice(16, seed=2)
    with crk.Sim(crk.box_physics(box), precision=0) as sim:
        sim.load(box)
        sim.forces(counts=False)
        pos = 0.5 + 0.75 * (box.pos - 0.5)
        crk.crk_set_state(sim.handle, pos, box.vel, box.u)
        out = sim.forces(counts=True)
    s = dict(box_dict(box), pos=pos)
    op = oracle_params(box)
    ref = oracle.forces(pos, box.vel, box.mass, box.u, box.h, box.species, op)
    assert ref["rc"] == 0
    compare(out, ref, oracle_counts(s, op), 0, label="compressed")


def test_pair_rows_beyond_capacity_walk_twice(crk):
    """A cut-off of most of the box gives every leaf more gravity leaf pairs
    than a fixed row holds: the lists are walked again (count, fill) and the
    gravity sets and forces still equal the oracle's."""
    box = wl.jittered_lattice(16, seed=5)
    params = dict(box.params(), r_cut=0.45, r_split=0.1)
    phys = crk.physics(**params)
    s = box_dict(box)
    op = oracle.make_params(**params)
    ref = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, op)
    assert ref["rc"] == 0
    with crk.Sim(phys, leaf_cap=32, precision=0) as sim:
        crk.crk_load(sim.handle, s["pos"], s["vel"], s["mass"], s["u"], s["h"], s["species"])
        sim.n = box.n
        out = sim.forces(counts=True)
        tim = crk.crk_get_timings(sim.handle)
    assert tim["pairs_grav"] > 256 * tim["nleaves"] // 2   # rows well beyond the fixed capacity
    compare(out, ref, oracle_counts(s, op), 0, label="wide cut-off")


# ------------------------------------------------------- pair-work census
def test_pair_census_of_one_leaf_is_exact(crk):
    """20 gas particles in one chaining-mesh cell, all within every cut-off:
    one leaf, one warp group of 20 targets, one visit that stages all 20
    candidates.  The census is then 32 x 20 lane slots per test pass, 20 x 20
    slots of lanes with a target, 400 list entries in 20 rows."""
    rng = np.random.default_rng(5)
    n = 20
    pos = 0.3125 + rng.uniform(-0.01, 0.01, (n, 3))
    phys = crk.physics(box=1.0, G=1.0, r_cut=0.1, r_split=0.02, eps_soft=0.001)
    with crk.Sim(phys, leaf_cap=32, precision=1) as sim:
        crk.crk_load(sim.handle, pos, np.zeros((n, 3)), np.full(n, 1e-3), np.ones(n), np.full(n, 0.03),
                     np.ones(n, np.uint8))
        sim.n = n
        t0 = crk.crk_get_timings(sim.handle)
        out = sim.forces(counts=True)
        t = crk.crk_get_timings(sim.handle)
    assert all(t0[k] == 0 for k in ("tests_hydro", "list_entries", "tests_grav", "tests_grav_target",
                                   "list_slots"))
    assert t["nleaves"] == 1
    assert np.all(out["nbr_count"] == n - 1) and np.all(out["grav_count"] == n - 1)
    assert (t["tests_hydro"], t["list_entries"], t["list_slots"]) == (32 * n, n * n, 32 * n)
    assert (t["tests_grav"], t["tests_grav_target"]) == (32 * n, n * n)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_pair_census_bounds_the_in_range_pairs(crk, precision):
    """Every in-range pair is tested once and written once: the tests cover
    the neighbour counts, the list entries hold at least the gather sets,
    the walked slots hold the entries; two counted evaluations test and write
    the same (the second one's rows are sized from the first one's counts
    with a margin, so it walks at least as many slots)."""
    box = wl.gaussian_field_box(16, seed=3)
    gas = box.species == wl.GAS
    with crk.Sim(crk.box_physics(box), precision=precision) as sim:
        sim.load(box)
        out = sim.forces(counts=True)
        t = crk.crk_get_timings(sim.handle)
        sim.forces(counts=True)
        t2 = crk.crk_get_timings(sim.handle)
    for k in ("tests_hydro", "list_entries", "tests_grav", "tests_grav_target"):
        assert t[k] == t2[k], k
    assert t2["list_slots"] >= t["list_slots"]
    gather = int(out["nbr_count"][gas].sum()) + int(gas.sum())    # self included
    grav = int(out["grav_count"].sum())
    assert t["list_entries"] >= gather
    assert t["tests_hydro"] >= t["list_entries"] and t["tests_hydro"] % 32 == 0
    assert t["list_slots"] >= t["list_entries"] and t["list_slots"] % 32 == 0
    assert t["tests_grav"] >= t["tests_grav_target"] >= grav + box.n
    assert t["tests_grav"] % 32 == 0
