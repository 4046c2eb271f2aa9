"""Pins of the oracle's long-range particle-mesh gravity against what the
mathematics fixes: the cloud-in-cell weights, a single Fourier mode solved in
closed form, momentum conservation, a uniform lattice, and the split itself
(the long-range pair force is the Newtonian one times 1 - S(r))."""
import math

import numpy as np
import pytest

from oracle import pm


def test_deposit_weights_and_mass():
    L, ng = 1.0, 8
    d = L / ng
    # at a cell centre: everything in that cell
    rho = pm.deposit(np.array([[2.5 * d, 3.5 * d, 4.5 * d]]), np.array([2.0]), L, ng)
    assert rho[2, 3, 4] == pytest.approx(2.0 / d ** 3, rel=1e-15)
    assert np.count_nonzero(rho) == 1
    # midway between 8 centres: an eighth each
    rho = pm.deposit(np.array([[3 * d, 3 * d, 3 * d]]), np.array([1.0]), L, ng)
    assert np.allclose(rho[2:4, 2:4, 2:4], 1.0 / 8 / d ** 3, rtol=1e-14)
    assert np.count_nonzero(rho) == 8
    # across the periodic face
    rho = pm.deposit(np.array([[0.0, 0.5 * d, 0.5 * d]]), np.array([1.0]), L, ng)
    assert rho[0, 0, 0] == pytest.approx(0.5 / d ** 3) and rho[ng - 1, 0, 0] == pytest.approx(0.5 / d ** 3)
    rng = np.random.default_rng(0)
    pos, m = rng.uniform(0, L, (500, 3)), rng.uniform(0.5, 1.5, 500)
    assert pm.deposit(pos, m, L, ng).sum() * d ** 3 == pytest.approx(m.sum(), rel=1e-13)


def test_interpolation_of_constant_and_linear_fields():
    L, ng = 1.0, 16
    d = L / ng
    rng = np.random.default_rng(1)
    pos = rng.uniform(0.2, 0.7, (300, 3))   # away from the periodic face
    const = np.ones((3, ng, ng, ng)) * np.array([1.0, -2.0, 3.0])[:, None, None, None]
    assert np.allclose(pm.interpolate(const, pos, L), [1.0, -2.0, 3.0], rtol=1e-14)
    c = (np.arange(ng) + 0.5) * d
    lin = np.broadcast_to(c[:, None, None], (ng, ng, ng))
    out = pm.interpolate(np.stack([lin, lin, lin]), pos, L)
    assert np.allclose(out[:, 0], pos[:, 0], atol=1e-14)


@pytest.mark.parametrize("m, axis", [(1, 0), (3, 1), (5, 2)])
def test_single_mode_has_the_closed_form(m, axis):
    L, ng, G, r_s = 2.0, 32, 1.7, 0.05
    d = L / ng
    c = (np.arange(ng) + 0.5) * d
    k = 2 * math.pi * m / L
    shape = [1, 1, 1]
    shape[axis] = ng
    rho = np.broadcast_to(np.cos(k * c).reshape(shape), (ng, ng, ng)).copy()
    acc = pm.solve(rho, L, G, r_s)
    C = np.sinc(k * d / 2 / np.pi) ** 2
    expect = -4 * math.pi * G / k * math.exp(-k * k * r_s * r_s) / C ** 2 * np.sin(k * c).reshape(shape)
    assert np.allclose(acc[axis], np.broadcast_to(expect, (ng, ng, ng)), rtol=1e-10, atol=1e-12)
    for other in range(3):
        if other != axis:
            assert np.max(np.abs(acc[other])) < 1e-10


def test_momentum_is_conserved():
    rng = np.random.default_rng(2)
    L, ng = 1.0, 32
    pos, m = rng.uniform(0, L, (2000, 3)), rng.uniform(0.5, 1.5, 2000)
    a = pm.accelerations(pos, m, L, ng, 1.0, 0.02)
    p = (m[:, None] * a).sum(0)
    scale = (m[:, None] * np.abs(a)).sum()
    assert np.max(np.abs(p)) < 1e-12 * scale


def test_uniform_lattice_feels_no_force():
    L, ng = 1.0, 16
    c = (np.arange(ng) + 0.5) * (L / ng)
    pos = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    a = pm.accelerations(pos, np.ones(len(pos)), L, ng, 1.0, 0.03)
    assert np.max(np.abs(a)) < 1e-10


def test_long_range_pair_force_is_newton_times_one_minus_S():
    """Two particles a few split scales apart in a large box: the mesh force
    on one is G m / r^2 (1 - S(r)) within the cloud-in-cell accuracy (a
    split of another width, e.g. exp(-k^2 r_s^2 / 2), is 4-23% off here)."""
    L, ng, G = 1.0, 128, 1.0
    d = L / ng
    r_s = 1.2 * d
    rng = np.random.default_rng(3)
    for r_over in (3.0, 4.0):
        r = r_over * r_s
        ratios = []
        for _ in range(12):
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            x0 = np.array([0.5, 0.5, 0.5]) + rng.uniform(-0.5, 0.5, 3) * d
            pos = np.stack([x0, x0 + r * u])
            a = pm.accelerations(pos, np.array([1.0, 1.0]), L, ng, G, r_s)
            ratios.append(np.dot(a[0], u))   # pull of particle 1 on particle 0, along u
        t = r / (2 * r_s)
        S = math.erfc(t) + r / (math.sqrt(math.pi) * r_s) * math.exp(-t * t)
        expect = G / r ** 2 * (1 - S)
        assert np.mean(ratios) == pytest.approx(expect, rel=0.01), r_over
