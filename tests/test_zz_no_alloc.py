"""The allocation-free neighbour-set entry point, for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or
cudaMalloc's implicit synchronisation is not acceptable in their loop).

Checked through the C ABI against the CPU oracle's neighbour sets and
against crk_forces' neighbour counts and hashes on the same box, on two calls
in a row (the calls share one static scratch array, so the second call must
not see stale state from the first).  This file is named to be collected
last.
"""
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


def _reference(crk, box):
    with crk.Sim(crk.box_physics(box), precision=crk.CRK_MIXED) as sim:
        sim.load(box)
        out = sim.forces(counts=True)
    return out["nbr_count"], out["nbr_hash"]


def _noalloc(crk, pos_np, h_np, sp_np, L):
    import torch

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    n = len(h_np)
    pos = torch.from_numpy(np.ascontiguousarray(pos_np)).to(dev)
    h = torch.from_numpy(np.ascontiguousarray(h_np)).to(dev)
    sp = torch.from_numpy(np.ascontiguousarray(sp_np)).to(dev)
    cnt = torch.full((n,), -7, dtype=torch.int32, device=dev)
    hs = torch.zeros(n, dtype=torch.int64, device=dev)
    rc = crk.lib().crk_neighbours_noalloc(
        crk.ctypes.c_int64(n), crk.ctypes.c_void_p(pos.data_ptr()),
        crk.ctypes.c_void_p(h.data_ptr()), crk.ctypes.c_void_p(sp.data_ptr()),
        crk.ctypes.c_double(L), crk.ctypes.c_void_p(cnt.data_ptr()),
        crk.ctypes.c_void_p(hs.data_ptr()), crk.ctypes.c_void_p(stream.cuda_stream))
    assert rc == crk.CRK_OK
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), hs.cpu().numpy().view(np.uint64)


def test_noalloc_neighbours_match_oracle_and_forces_on_two_calls(crk):
    boxes = [wl.jittered_lattice(16, seed=3), wl.gaussian_field_box(24, seed=5)]
    for box in boxes:
        op = oracle.make_params(**box.params())
        orc_c, orc_h = oracle.neighbours(box.pos, box.h, box.species, op, 0)
        ref_c, ref_h = _reference(crk, box)
        for _ in range(2):
            c, h = _noalloc(crk, box.pos, box.h, box.species, box.L)
            assert np.array_equal(c, orc_c) and np.array_equal(h, orc_h)
            assert np.array_equal(c, ref_c) and np.array_equal(h, ref_h)


def test_noalloc_cells_when_the_box_is_a_whole_number_of_supports(crk):
    """box / max(2h) = 5 exactly (h = 0.1): gas pairs placed just inside the
    support across the cell faces are all found, as the oracle finds them."""
    rng = np.random.default_rng(9)
    base = rng.uniform(0, 1, size=(400, 3))
    near = []
    for k in range(1, 6):
        for axis in range(3):
            a = rng.uniform(0.05, 0.95, 3)
            a[axis] = 0.2 * k - 1e-12
            b = a.copy()
            b[axis] = a[axis] + (0.2 - 3e-12)      # r just below 2h, across a cell face
            near += [a, b]
    pos = np.concatenate([base, np.array(near) % 1.0])
    pos[pos >= 1.0] = 0.0
    n = len(pos)
    sp = np.ones(n, np.uint8)
    h = np.full(n, 0.1)
    op = oracle.make_params(box=1.0, r_cut=0.2)
    orc_c, orc_h = oracle.neighbours(pos, h, sp, op, 0)
    for _ in range(2):
        c, hs = _noalloc(crk, pos, h, sp, 1.0)
        assert np.array_equal(c, orc_c) and np.array_equal(hs, orc_h)


def test_noalloc_reports_invalid_particles(crk):
    """A position outside [0, box) and a gas h that is not finite give count
    -1 for those particles; the others' sets equal the oracle's with the
    misplaced particle taken out of every set."""
    box = wl.gaussian_field_box(12, seed=6)
    pos, h, sp = box.pos.copy(), box.h.copy(), box.species.copy()
    gas = np.flatnonzero(sp == wl.GAS)
    bad_pos, bad_h = gas[3], gas[10]
    pos[bad_pos, 1] = 1.5
    h[bad_h] = np.nan
    c, hs = _noalloc(crk, pos, h, sp, box.L)
    assert c[bad_pos] == -1 and hs[bad_pos] == 0
    assert c[bad_h] == -1 and hs[bad_h] == 0
    # the oracle on the valid particles: the misplaced one is made DM (in no
    # gas set), the NaN-h one keeps a valid h (its own set is not compared)
    sp2, h2, pos2 = sp.copy(), box.h.copy(), box.pos.copy()
    sp2[bad_pos] = wl.DM
    op = oracle.make_params(**box.params())
    orc_c, orc_h = oracle.neighbours(pos2, h2, sp2, op, 0)
    keep = np.ones(box.n, bool)
    keep[[bad_pos, bad_h]] = False
    assert np.array_equal(c[keep], orc_c[keep]) and np.array_equal(hs[keep], orc_h[keep])


def test_noalloc_rejects_sizes_beyond_its_maximum(crk):
    import torch

    dev = torch.device("cuda", 0)
    n = crk.CRK_NOALLOC_MAX_N + 1
    buf = torch.zeros(1, dtype=torch.float64, device=dev)
    p = crk.ctypes.c_void_p(buf.data_ptr())
    rc = crk.lib().crk_neighbours_noalloc(crk.ctypes.c_int64(n), p, p, p, crk.ctypes.c_double(1.0),
                                          p, p, None)
    assert rc == crk.CRK_EINVAL
