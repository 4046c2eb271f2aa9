"""The allocation-free neighbour-set entry point, for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or
cudaMalloc's implicit synchronisation is not acceptable in their loop).

Checked through the C ABI against crk_forces' neighbour counts and hashes on
the same box, on two calls in a row (the calls share one static scratch
array, so the second call must not see stale state from the first).  This
file is named to be collected last.
"""
import numpy as np
import pytest

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


def test_noalloc_neighbours_match_forces_on_two_calls(crk):
    import torch

    dev = torch.device("cuda", 0)
    boxes = [wl.jittered_lattice(16, seed=3), wl.gaussian_field_box(24, seed=5)]
    stream = torch.cuda.current_stream()
    for box in boxes:
        ref_c, ref_h = _reference(crk, box)
        pos = torch.from_numpy(np.ascontiguousarray(box.pos)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(box.h)).to(dev)
        sp = torch.from_numpy(np.ascontiguousarray(box.species)).to(dev)
        for _ in range(2):
            cnt = torch.full((box.n,), -1, dtype=torch.int32, device=dev)
            hs = torch.zeros(box.n, dtype=torch.int64, device=dev)
            rc = crk.lib().crk_neighbours_noalloc(
                crk.ctypes.c_int64(box.n), crk.ctypes.c_void_p(pos.data_ptr()),
                crk.ctypes.c_void_p(h.data_ptr()), crk.ctypes.c_void_p(sp.data_ptr()),
                crk.ctypes.c_double(box.L), crk.ctypes.c_void_p(cnt.data_ptr()),
                crk.ctypes.c_void_p(hs.data_ptr()), crk.ctypes.c_void_p(stream.cuda_stream))
            assert rc == crk.CRK_OK
            torch.cuda.synchronize()
            assert np.array_equal(cnt.cpu().numpy(), ref_c)
            assert np.array_equal(hs.cpu().numpy().view(np.uint64), ref_h)


def test_noalloc_rejects_sizes_beyond_its_maximum(crk):
    import torch

    dev = torch.device("cuda", 0)
    n = crk.CRK_NOALLOC_MAX_N + 1
    buf = torch.zeros(1, dtype=torch.float64, device=dev)
    p = crk.ctypes.c_void_p(buf.data_ptr())
    rc = crk.lib().crk_neighbours_noalloc(crk.ctypes.c_int64(n), p, p, p, crk.ctypes.c_double(1.0),
                                          p, p, None)
    assert rc == crk.CRK_EINVAL
