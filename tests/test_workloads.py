"""The seeded input generators against the input recipe: lattices, masses,
the curl-free k^-2 displacement field and its rms, velocities, log-normal
energies, Plummer spheres and kNN smoothing lengths (by brute force), the
time-step rule, the serving sizes and the batched boxes."""
import math

import numpy as np
import pytest

from paper_2510_03557_gb300 import workloads as wl


def _periodic(d):
    return (d + 0.5) % 1.0 - 0.5


def _lattice(n, off):
    g = (np.arange(n) + off) / n
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


def test_jittered_lattice_recipe():
    n = 8
    b = wl.jittered_lattice(n, seed=3)
    n3 = n ** 3
    assert b.n == 2 * n3 and np.all(b.species[:n3] == wl.DM) and np.all(b.species[n3:] == wl.GAS)
    assert np.all((b.pos >= 0) & (b.pos < 1))
    assert np.max(np.abs(_periodic(b.pos[:n3] - _lattice(n, 0.0)))) <= 0.1 / n
    assert np.max(np.abs(_periodic(b.pos[n3:] - _lattice(n, 0.5)))) <= 0.1 / n
    assert b.mass[:n3].sum() == pytest.approx(0.84) and b.mass[n3:].sum() == pytest.approx(0.16)
    assert np.all(b.vel == 0) and np.all(b.u[n3:] == 1) and np.all(b.u[:n3] == 0)
    assert np.all(b.h[n3:] == 2.0 / n)
    assert b.r_cut == pytest.approx(3.0 / n) and b.r_split == pytest.approx(b.r_cut / 4.5)
    assert b.eps_soft == pytest.approx(0.05 / n)
    exact = wl.jittered_lattice(n, seed=3, jitter=0.0)
    assert np.allclose(exact.pos[n3:], _lattice(n, 0.5), atol=1e-15)


def test_gaussian_field_recipe():
    n = 16
    b = wl.gaussian_field_box(n, seed=7)
    n3 = n ** 3
    d_dm = _periodic(b.pos[:n3] - _lattice(n, 0.0))
    d_gas = _periodic(b.pos[n3:] - _lattice(n, 0.5))
    rms = lambda d: math.sqrt(float(np.mean(np.sum(d * d, axis=1))))
    # 0.3-cell 3-D rms on both lattices (the half-cell phase shift keeps the power)
    assert rms(d_dm) == pytest.approx(0.3 / n, rel=1e-9)
    assert rms(d_gas) == pytest.approx(0.3 / n, rel=1e-9)
    assert np.allclose(b.vel[:n3], 0.5 * d_dm, atol=1e-15)
    assert np.allclose(b.vel[n3:], 0.5 * d_gas, atol=1e-15)
    # curl-free, and nothing at or above the Nyquist wavenumber
    D = np.stack([np.fft.fftn(d_dm[:, a].reshape(n, n, n)) for a in range(3)], -1)
    k1 = 2 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    K = np.stack(np.meshgrid(k1, k1, k1, indexing="ij"), -1)
    cross = np.cross(K, D)
    kk = np.linalg.norm(K, axis=-1)
    dd = np.linalg.norm(D, axis=-1)
    assert np.max(np.abs(cross)) <= 1e-9 * np.max(kk * dd)
    assert np.max(dd[kk >= np.pi * n]) <= 1e-12 * np.max(dd)
    # |psi(k)|^2 k^2 is the white noise's power: flat in k on average
    keep = (kk > 0) & (kk < np.pi * n)
    p = (dd ** 2 * kk ** 2)[keep]
    lo, hi = kk[keep] < np.median(kk[keep]), kk[keep] >= np.median(kk[keep])
    assert p[lo].mean() / p[hi].mean() == pytest.approx(1.0, abs=0.1)
    # log-normal u with median 1 and sigma 0.5 for the gas, zero for DM
    lu = np.log(b.u[n3:])
    assert abs(lu.mean()) < 4 * 0.5 / math.sqrt(n3) and lu.std() == pytest.approx(0.5, rel=0.05)
    assert np.all(b.u[:n3] == 0)
    assert b.dt == 1e-3 and b.nsteps == 10 and np.all(b.h[n3:] == 2.0 / n)


def test_clustered_recipe_and_knn_h_by_brute_force():
    n, nsphere, a = 12, 8, 0.002
    b = wl.clustered_box(n, seed=9, nsphere=nsphere, a=a)
    n3 = n ** 3
    per = (n3 - n3 // 2) // nsphere
    nuni = n3 - nsphere * per
    gas = b.species == wl.GAS
    for s in (wl.DM, wl.GAS):
        p = b.pos[b.species == s]
        cl = p[nuni:].reshape(nsphere, per, 3)
        for k in range(nsphere):
            r = np.linalg.norm(_periodic(cl[k] - cl[k][0]), axis=1)
            assert np.max(r) <= 2 * 20 * a + 1e-12          # truncated at 20a around a shared centre
    # both species share the sphere centres
    dm_cl = b.pos[:n3][nuni:].reshape(nsphere, per, 3)
    gas_cl = b.pos[n3:][nuni:].reshape(nsphere, per, 3)
    for k in range(nsphere):
        assert np.linalg.norm(_periodic(dm_cl[k][0] - gas_cl[k][0])) <= 2 * 20 * a + 1e-12
    # h = 1.2 x the distance to the 32nd-nearest other gas particle (brute force, periodic)
    g = b.pos[gas]
    d = np.linalg.norm(_periodic(g[:, None, :] - g[None, :, :]), axis=-1)
    np.fill_diagonal(d, np.inf)
    want = 1.2 * np.sort(d, axis=1)[:, 31]
    assert np.allclose(b.h[gas], want, rtol=1e-12)
    # the time step: a quarter of the smallest h / c, one significant digit, at most 1e-4
    c = np.sqrt((5 / 3) * (2 / 3) * b.u[gas])
    x = 0.25 * np.min(b.h[gas] / c)
    e = math.floor(math.log10(x))
    assert b.dt == pytest.approx(min(1e-4, math.floor(x / 10 ** e) * 10 ** e))
    assert np.all(b.vel == 0) and b.nsteps == 5


def test_serving_sizes_are_log_uniform():
    reqs = wl.serving_requests()
    ns = np.array([r[0] for r in reqs])
    assert len(reqs) == 2000 and ns.min() >= 16 and ns.max() <= 128
    assert [r[1] for r in reqs[:3]] == [10000, 10001, 10002]
    # E[n^3] for log-uniform n in [16, 128] = (128^3 - 16^3) / (3 ln 8) = 335,540
    assert np.mean(ns.astype(float) ** 3) == pytest.approx((128 ** 3 - 16 ** 3) / (3 * math.log(8)), rel=0.15)
    # log n is uniform: its quartiles sit at the quarter points of [ln 16, ln 128]
    q = np.quantile(np.log(ns), [0.25, 0.5, 0.75])
    lo, hi = math.log(16), math.log(128)
    assert np.allclose(q, [lo + f * (hi - lo) for f in (0.25, 0.5, 0.75)], atol=0.1)


def test_batched_boxes_are_gaussian_field_boxes():
    boxes = wl.batched_boxes(nbox=5, sizes=(6, 8))
    for k, bx in enumerate(boxes):
        ref = wl.gaussian_field_box(bx.n_lattice, seed=1000 + k)
        assert bx.n_lattice in (6, 8) and np.array_equal(bx.pos, ref.pos) and np.array_equal(bx.u, ref.u)
    cat = wl.concat_boxes(boxes)
    assert list(cat["offsets"]) == list(np.cumsum([0] + [bx.n for bx in boxes]))


def test_poisson_arrivals():
    t = wl.poisson_arrivals(4000, rate_per_s=2.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and gaps.mean() == pytest.approx(0.5, rel=0.06)
    assert gaps.std() == pytest.approx(0.5, rel=0.08)   # exponential: sd = mean
