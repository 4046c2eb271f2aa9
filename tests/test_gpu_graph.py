"""Steps replayed from a CUDA graph (crk_step with nsteps >= 3): every size
stays on the device, the pair passes drain a device work queue.  Checked
against host-sized steps of the same handle type (CRK_FLAG_NO_GRAPH) and the
oracle's KDK; the overflow path (a flow that outgrows the capacities of the
first step) restores and reruns; the step counters show that replayed steps
synchronise with the host only once per call."""
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


def rel_l2(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def disp_err(pos, ref, pos0):
    d = (pos - ref + 0.5) % 1.0 - 0.5
    return np.linalg.norm(d) / np.linalg.norm((ref - pos0 + 0.5) % 1.0 - 0.5)


def _run(crk, box, precision, nsteps, flags=0, stream=None, margin=0):
    import torch

    st = stream or torch.cuda.Stream()
    with crk.Sim(crk.box_physics(box), leaf_cap=64, precision=precision, stream=st, flags=flags,
                 graph_margin_pct=margin) as sim:
        sim.load(box)
        crk.crk_set_timing(sim.handle, False)
        sim.step(box.dt, nsteps)
        t = crk.crk_get_timings(sim.handle)
        pos, vel, u = sim.state()
    return pos, vel, u, t


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_replayed_steps_match_host_sized_steps_and_the_oracle(crk, precision):
    box = wl.gaussian_field_box(16, seed=71)
    box.vel = box.vel * 20.0
    nsteps = 7
    g = _run(crk, box, precision, nsteps)
    e = _run(crk, box, precision, nsteps, flags=crk.CRK_FLAG_NO_GRAPH)
    # 1 host-sized step, then 3 replays of two steps
    assert g[3]["steps"] == nsteps and g[3]["graph_steps"] == 6 and g[3]["graph_overflows"] == 0
    assert e[3]["graph_steps"] == 0
    # the host-sized step synchronises several times, a replay batch once
    assert g[3]["host_syncs"] < e[3]["host_syncs"] / 3
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species,
                     oracle.make_params(**box.params()), box.dt, nsteps)
    tol = 1e-10 if precision == 0 else 2e-4
    for r in (g, e):
        assert disp_err(r[0], ref["pos"], box.pos) <= tol
        assert rel_l2(r[1], ref["vel"]) <= tol and rel_l2(r[2], ref["u"]) <= tol
    same = 1e-12 if precision == 0 else 1e-5
    assert disp_err(g[0], e[0], box.pos) <= same and rel_l2(g[1], e[1]) <= same


def test_replayed_steps_with_pairs_once_forms_match_the_oracle(crk):
    """The mixed form with gravity and hydro pairs evaluated once (the rates
    zeroed and accumulated by atomics inside the captured graph)."""
    box = wl.gaussian_field_box(16, seed=74)
    box.vel = box.vel * 20.0
    flags = crk.CRK_FLAG_GRAVITY_PAIRS_ONCE | crk.CRK_FLAG_HYDRO_PAIRS_ONCE
    g = _run(crk, box, 1, 7, flags=flags)
    assert g[3]["graph_steps"] == 6 and g[3]["graph_overflows"] == 0
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species,
                     oracle.make_params(**box.params()), box.dt, 7)
    assert disp_err(g[0], ref["pos"], box.pos) <= 2e-4
    assert rel_l2(g[1], ref["vel"]) <= 2e-4 and rel_l2(g[2], ref["u"]) <= 2e-4


def test_replayed_steps_of_batched_boxes_match_the_oracle(crk):
    import torch

    boxes = [wl.gaussian_field_box(n, seed=720 + n) for n in (10, 16, 12)]
    cat = wl.concat_boxes(boxes)
    phys = [crk.box_physics(b) for b in boxes]
    dts = [1e-3, 2e-3, 1.5e-3]
    nsteps = 5
    with crk.Sim(phys[0], precision=0, stream=torch.cuda.Stream()) as sim:
        crk.crk_load_boxes(sim.handle, [b.n for b in boxes], phys, cat["pos"], cat["vel"], cat["mass"],
                           cat["u"], cat["h"], cat["species"])
        crk.crk_set_timing(sim.handle, False)
        crk.crk_step_boxes(sim.handle, dts, nsteps)
        t = crk.crk_get_timings(sim.handle)
        n = int(cat["offsets"][-1])
        pos, vel, u = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
        crk.crk_get_state(sim.handle, pos, vel, u)
    assert t["graph_steps"] == 4
    for b, box in enumerate(boxes):
        lo, hi = cat["offsets"][b], cat["offsets"][b + 1]
        ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species,
                         oracle.make_params(**box.params()), dts[b], nsteps)
        assert rel_l2(vel[lo:hi], ref["vel"]) <= 1e-10
        assert rel_l2(u[lo:hi], ref["u"]) <= 1e-10


def test_replays_that_outgrow_their_capacities_run_again(crk):
    """A converging flow compresses the box (the gather sets grow by about
    60% over the steps), so the hydro lists outgrow the capacities of the
    first step (taken with a 1% margin): the batch is restored and stepped
    host-sized, and the result is still the oracle's."""
    box = wl.jittered_lattice(16, seed=12)
    d = (box.pos - 0.5 + 0.5) % 1.0 - 0.5
    box.vel = -15.0 * d
    box.dt = 2e-3
    nsteps = 9
    g = _run(crk, box, 0, nsteps, margin=1)
    assert g[3]["graph_overflows"] >= 1 and g[3]["steps"] == nsteps
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species,
                     oracle.make_params(**box.params()), box.dt, nsteps)
    assert disp_err(g[0], ref["pos"], box.pos) <= 1e-10
    assert rel_l2(g[1], ref["vel"]) <= 1e-10


def test_handles_on_the_default_stream_replay_too(crk):
    box = wl.gaussian_field_box(12, seed=73)
    with crk.Sim(crk.box_physics(box), precision=1) as sim:      # legacy default stream
        sim.load(box)
        crk.crk_set_timing(sim.handle, False)
        sim.step(box.dt, 5)
        t = crk.crk_get_timings(sim.handle)
        pos, vel, u = sim.state()
    assert t["graph_steps"] == 4
    ref = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species,
                     oracle.make_params(**box.params()), box.dt, 5)
    assert rel_l2(vel, ref["vel"]) <= 2e-4
