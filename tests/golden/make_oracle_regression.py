"""Writes oracle_regression.json: the CPU oracle's outputs on two small seeded
boxes (norms per output, and every output of eight particles), so that any
later change to the oracle's arithmetic shows up in
tests/test_oracle_regression.py.  Calls only ``oracle`` and the input
generators.  Run from the repository root:

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2510_03557_gb300 import workloads as wl  # noqa: E402

OUTPUTS = ("acc", "dudt", "rho", "A", "B", "dA", "dB")


def sample(box):
    """Eight particles: DM and gas, first, last and in between."""
    n3 = box.n // 2
    return [0, 1, 17, n3 // 3, n3 - 1, n3, n3 + n3 // 2, 2 * n3 - 1]


def cases():
    g = wl.gaussian_field_box(12, seed=31)
    g.vel = g.vel * 20.0
    c = wl.clustered_box(20, seed=32, nsphere=16)
    for b in (g, c):  # the solver's precondition max(2h, r_cut) < L/2
        assert max(2.0 * b.h.max(), b.r_cut) < 0.5 * b.L
    return {"gaussian_2x12": g, "clustered_2x20": c}


def evaluate(box):
    p = oracle.make_params(**box.params())
    r = oracle.forces(box.pos, box.vel, box.mass, box.u, box.h, box.species, p)
    assert r["rc"] == 0
    k = oracle.kdk(box.pos, box.vel, box.mass, box.u, box.h, box.species, p, 1e-4, 2)
    out = {"norm_" + o: float(np.linalg.norm(r[o])) for o in OUTPUTS}
    idx = sample(box)
    out.update({"sample_" + o: np.asarray(r[o])[idx].tolist() for o in OUTPUTS})
    out.update({"kdk_norm_vel": float(np.linalg.norm(k["vel"])), "kdk_norm_u": float(np.linalg.norm(k["u"])),
                "kdk_sample_pos": np.asarray(k["pos"])[idx].tolist()})
    return out


def main():
    oracle.build()
    data = {name: evaluate(box) for name, box in cases().items()}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(data, f, indent=1)


if __name__ == "__main__":
    main()
