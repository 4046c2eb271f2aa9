"""Seeded synthetic particle sets shaped like the paper's workloads.

This module only draws inputs.  It contains none of the method's arithmetic
(no smoothing kernel, no pair sums, no corrections): it places particles,
assigns masses, velocities, thermal energies and smoothing lengths, and
returns plain NumPy arrays that feed both the CUDA path and the CPU oracle.

The paper's production workload (Sec. II and Sec. V, Frontier-E) is a
cosmological volume with equal numbers of dark-matter and gas particles and
about 270 neighbours per CRKSPH evaluation (Sec. IV-B1).  Its initial
conditions are not available, so the generators below are stand-ins with the
same species split, neighbour count and (for the clustered case) a strongly
inhomogeneous density.

Species codes: 0 = dark matter (gravity only), 1 = gas.
All boxes are periodic with side ``L`` = 1 unless stated.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DM = 0
GAS = 1


@dataclasses.dataclass
class Box:
    """One periodic box of particles (arrays in the caller's order)."""

    pos: np.ndarray       # (N, 3) float64 in [0, L)
    vel: np.ndarray       # (N, 3) float64
    mass: np.ndarray      # (N,) float64
    u: np.ndarray         # (N,) float64 specific thermal energy (gas; 0 for DM)
    h: np.ndarray         # (N,) float64 smoothing length (gas; DM entries unused)
    species: np.ndarray   # (N,) uint8, 0 = DM, 1 = gas
    L: float = 1.0
    G: float = 1.0
    gamma: float = 5.0 / 3.0
    r_cut: float = 0.0
    r_split: float = 0.0
    eps_soft: float = 0.0
    dt: float = 0.0
    nsteps: int = 0
    n_lattice: int = 0
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def params(self) -> dict:
        return dict(box=self.L, G=self.G, gamma=self.gamma, r_cut=self.r_cut,
                    r_split=self.r_split, eps_soft=self.eps_soft)


def _wrap(x: np.ndarray, L: float) -> np.ndarray:
    """Map coordinates into [0, L) (a placement step, not part of the method)."""
    x = np.mod(x, L)
    x[x >= L] = 0.0
    return x


def _lattice(n: int, offset: float) -> np.ndarray:
    g = (np.arange(n, dtype=np.float64) + offset) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _gravity_scales(n: int, box: Box) -> None:
    """Short-range gravity constants tied to an n^3 PM grid: cut-off 3 cells,
    Gaussian split scale r_cut / 4.5 and Plummer-equivalent softening of
    0.05 of the mean inter-particle spacing."""
    box.r_cut = 3.0 / n
    box.r_split = box.r_cut / 4.5
    box.eps_soft = 0.05 / n


def jittered_lattice(n: int = 32, seed: int = 0, jitter: float = 0.1) -> Box:
    """Two interleaved n^3 lattices (DM at cell corners, gas at cell centres)
    with every coordinate displaced by U(-jitter, +jitter) cells.  Total mass
    0.84 in DM and 0.16 in gas, v = 0, u = 1, h = 2 mean gas spacings."""
    rng = np.random.default_rng(seed)
    n3 = n ** 3
    dm = _lattice(n, 0.0)
    gas = _lattice(n, 0.5)
    pos = np.concatenate([dm, gas])
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) / n
    pos = _wrap(pos, 1.0)
    species = np.concatenate([np.full(n3, DM, np.uint8), np.full(n3, GAS, np.uint8)])
    mass = np.where(species == GAS, 0.16 / n3, 0.84 / n3).astype(np.float64)
    u = np.where(species == GAS, 1.0, 0.0)
    h = np.where(species == GAS, 2.0 / n, 0.0)
    box = Box(pos=pos, vel=np.zeros_like(pos), mass=mass, u=u, h=h, species=species,
              n_lattice=n, name=f"jittered-lattice-2x{n}^3")
    _gravity_scales(n, box)
    return box


def _displacement_field(n: int, rng: np.random.Generator, rms_cells: float):
    """Curl-free Gaussian displacement psi(k) = i k_hat s(k) / k from white
    noise s, so |psi(k)|^2 ~ k^-2, with every mode at or above the n^3 Nyquist
    wavenumber removed.  Returns the field sampled on the DM lattice and on
    the gas lattice (the latter through an exact half-cell Fourier phase
    shift), scaled so the 3-D rms displacement is ``rms_cells`` cells."""
    s = rng.standard_normal((n, n, n))
    S = np.fft.fftn(s)
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k_nyq = np.pi * n
    keep = (k2 > 0) & (k2 < k_nyq ** 2)
    inv_k2 = np.zeros_like(k2)
    inv_k2[keep] = 1.0 / k2[keep]
    shift = np.exp(1j * (KX + KY + KZ) * (0.5 / n))
    fields = []
    for phase in (1.0, shift):
        comps = []
        for K in (KX, KY, KZ):
            psi_k = 1j * K * inv_k2 * S * phase
            comps.append(np.real(np.fft.ifftn(psi_k)))
        fields.append(np.stack([c.ravel() for c in comps], axis=1))
    rms = math.sqrt(float(np.mean(np.sum(fields[0] ** 2, axis=1))))
    scale = (rms_cells / n) / rms if rms > 0 else 0.0
    return fields[0] * scale, fields[1] * scale


def gaussian_field_box(n: int = 128, seed: int = 1, rms_cells: float = 0.3,
                       u_sigma: float = 0.5) -> Box:
    """Two n^3 lattices displaced by a P(k) ~ k^-2 Gaussian random field of
    0.3-cell rms, velocities 0.5 x displacement, log-normal gas u (median 1),
    fixed h = 2 mean gas spacings; 10 KDK steps at dt = 1e-3."""
    rng = np.random.default_rng(seed)
    n3 = n ** 3
    psi_dm, psi_gas = _displacement_field(n, rng, rms_cells)
    dm = _lattice(n, 0.0) + psi_dm
    gas = _lattice(n, 0.5) + psi_gas
    pos = _wrap(np.concatenate([dm, gas]), 1.0)
    vel = 0.5 * np.concatenate([psi_dm, psi_gas])
    species = np.concatenate([np.full(n3, DM, np.uint8), np.full(n3, GAS, np.uint8)])
    mass = np.where(species == GAS, 0.16 / n3, 0.84 / n3).astype(np.float64)
    u = np.zeros(2 * n3)
    u[n3:] = np.exp(rng.normal(0.0, u_sigma, size=n3))
    h = np.where(species == GAS, 2.0 / n, 0.0)
    box = Box(pos=pos, vel=vel, mass=mass, u=u, h=h, species=species,
              dt=1e-3, nsteps=10, n_lattice=n, name=f"gaussian-field-2x{n}^3")
    _gravity_scales(n, box)
    return box


BATCH_SIZES = (16, 24, 32, 48, 64)


def batched_boxes(nbox: int = 64, seed: int = 2, sizes=BATCH_SIZES) -> list[Box]:
    """``nbox`` independent periodic boxes, each 2 x n^3 particles with n drawn
    (seeded) from ``sizes``, box b built by the Gaussian-field generator with
    seed 1000 + b."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=nbox)
    return [gaussian_field_box(int(n), seed=1000 + b) for b, n in enumerate(ns)]


def _plummer_offsets(rng: np.random.Generator, count: int, a: float, rmax_over_a: float):
    """Radii from the Plummer cumulative mass profile, truncated at rmax."""
    x = rmax_over_a
    m_max = x ** 3 / (1.0 + x * x) ** 1.5
    U = rng.uniform(0.0, m_max, size=count)
    U = np.maximum(U, 1e-300)
    r = a / np.sqrt(U ** (-2.0 / 3.0) - 1.0)
    v = rng.standard_normal((count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * r[:, None]


def knn_smoothing_lengths(gas_pos: np.ndarray, k: int = 32, factor: float = 1.2,
                          L: float = 1.0) -> np.ndarray:
    """h_i = factor x distance to the k-th nearest *other* gas particle
    (periodic).  This is an input-placement step done once at set-up with a
    library k-d tree; the method itself receives h as an input."""
    from scipy.spatial import cKDTree

    tree = cKDTree(gas_pos, boxsize=L)
    d, _ = tree.query(gas_pos, k=k + 1, workers=-1)
    return factor * d[:, k]


def _round_down_1sig(x: float) -> float:
    """x rounded down to one significant decimal digit."""
    e = math.floor(math.log10(x))
    return math.floor(x / 10.0 ** e) * 10.0 ** e


def clustered_box(n: int = 256, seed: int = 3, nsphere: int = 512, a: float = 0.002,
                  u_sigma: float = 1.0, knn: bool = True) -> Box:
    """2 x n^3 particles; per species half uniform and half in ``nsphere``
    Plummer spheres (scale radius ``a``, truncated at 20a, centres uniform and
    shared by both species, equal split per sphere); v = 0; log-normal gas u
    (median 1, sigma 1); adaptive h from the 32nd-nearest gas neighbour;
    one force evaluation plus 5 KDK steps.  The step is a Courant bound of the
    initial state, dt = 0.25 min_gas h / c with c = sqrt(gamma (gamma-1) u),
    rounded down to one significant digit and at most 1e-4 (2x256^3: 8e-6);
    a fixed 1e-4 moves the densest core particles by several h per step."""
    rng = np.random.default_rng(seed)
    n3 = n ** 3
    half = n3 // 2
    per = (n3 - half) // nsphere
    centres = rng.uniform(0.0, 1.0, size=(nsphere, 3))
    parts = []
    for _sp in (DM, GAS):
        uni = rng.uniform(0.0, 1.0, size=(n3 - nsphere * per, 3))
        cl = np.repeat(centres, per, axis=0) + _plummer_offsets(rng, nsphere * per, a, 20.0)
        parts.append(_wrap(np.concatenate([uni, cl]), 1.0))
    pos = np.concatenate(parts)
    species = np.concatenate([np.full(n3, DM, np.uint8), np.full(n3, GAS, np.uint8)])
    mass = np.where(species == GAS, 0.16 / n3, 0.84 / n3).astype(np.float64)
    u = np.zeros(2 * n3)
    u[n3:] = np.exp(rng.normal(0.0, u_sigma, size=n3))
    h = np.zeros(2 * n3)
    if knn:
        h[n3:] = knn_smoothing_lengths(pos[n3:], 32, 1.2)
    else:
        h[n3:] = 2.0 / n
    gas = species == GAS
    c = np.sqrt((5.0 / 3.0) * (2.0 / 3.0) * u[gas])
    dt = min(1e-4, _round_down_1sig(0.25 * float(np.min(h[gas] / c))))
    box = Box(pos=pos, vel=np.zeros_like(pos), mass=mass, u=u, h=h, species=species,
              dt=dt, nsteps=5, n_lattice=n, name=f"clustered-2x{n}^3")
    _gravity_scales(n, box)
    return box


def serving_requests(count: int = 2000, seed: int = 4, nmin: int = 16, nmax: int = 128):
    """Request sizes for the serving workload: n log-uniform in [nmin, nmax]
    (rounded), each box built later by the Gaussian-field generator with the
    per-request seed 10000 + index; 20 KDK steps at dt = 1e-3."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(int)
    return [(int(n), 10000 + i) for i, n in enumerate(ns)]


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Arrival offsets (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def concat_boxes(boxes: list[Box]):
    """Flatten a list of boxes into one particle set with a per-particle box
    index and per-box offsets (placement bookkeeping only)."""
    offs = np.zeros(len(boxes) + 1, dtype=np.int64)
    for b, bx in enumerate(boxes):
        offs[b + 1] = offs[b] + bx.n
    cat = lambda f: np.concatenate([getattr(bx, f) for bx in boxes])
    return dict(pos=cat("pos"), vel=cat("vel"), mass=cat("mass"), u=cat("u"), h=cat("h"),
                species=cat("species"), offsets=offs)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014), used to hash
    neighbour identities order-independently.  Published definition:
    z = x + 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
    z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))
