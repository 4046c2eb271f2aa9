"""Long-range particle-mesh gravity of the long/short split: plain FP64 numpy.

TEST INFRASTRUCTURE.  Only the test suite loads this module; the product
path never calls it and shares no code with it.

The paper evaluates the long-range part of gravity with a spectral
particle-mesh solver in FP64 (Sec. IV-A) and leaves the short-range part to
the particle-particle solver; the split and the filter are cited, not
printed.  Reading (the Gaussian split whose short-range factor is
S(r) = erfc(r / 2 r_s) + r / (sqrt(pi) r_s) exp(-r^2 / 4 r_s^2)): the
long-range potential is the Newtonian one filtered by exp(-k^2 r_s^2), so
that long + short is Newtonian for every pair.  Steps, for particles in a
periodic cube of side L on an n_g^3 mesh of cell d = L / n_g:

  1. cloud-in-cell deposit: rho_g = sum_p m_p W(x_p - x_g) / d^3 with the
     linear weights W of the 8 cells around x_p (cell centres at (i + 1/2) d);
  2. rho(k) = FFT(rho_g);
  3. phi(k) = -4 pi G rho(k) exp(-k^2 r_s^2) / (k^2 C(k)^2), phi(0) = 0, where
     C(k) = prod_a sinc^2(k_a d / 2) undoes the deposit and the interpolation
     windows (sinc x = sin x / x);
  4. a(k) = -i k phi(k), the derivative of the Nyquist plane of each axis set
     to zero (a real field's odd derivative there is not defined);
  5. a_g = inverse FFT, then the same cloud-in-cell weights interpolate a_g
     back to every particle.
"""
from __future__ import annotations

import numpy as np


def cic_weights(pos: np.ndarray, L: float, ng: int):
    """For every particle the 8 cells (flat indices) and weights of the
    cloud-in-cell assignment (cell centres at (i + 1/2) L / ng)."""
    d = L / ng
    s = pos / d - 0.5                      # position in units of cells, from the first centre
    i0 = np.floor(s).astype(np.int64)
    f = s - i0                             # fraction towards the next centre
    cells, weights = [], []
    for ox in (0, 1):
        wx = f[:, 0] if ox else 1.0 - f[:, 0]
        for oy in (0, 1):
            wy = f[:, 1] if oy else 1.0 - f[:, 1]
            for oz in (0, 1):
                wz = f[:, 2] if oz else 1.0 - f[:, 2]
                ix = (i0[:, 0] + ox) % ng
                iy = (i0[:, 1] + oy) % ng
                iz = (i0[:, 2] + oz) % ng
                cells.append((ix * ng + iy) * ng + iz)
                weights.append(wx * wy * wz)
    return np.stack(cells, 1), np.stack(weights, 1)


def deposit(pos, mass, L: float, ng: int) -> np.ndarray:
    """Step 1: mass density on the mesh, shape (ng, ng, ng), index [x, y, z]."""
    cells, w = cic_weights(np.asarray(pos, np.float64), L, ng)
    rho = np.zeros(ng ** 3)
    np.add.at(rho, cells.ravel(), (w * np.asarray(mass, np.float64)[:, None]).ravel())
    return rho.reshape(ng, ng, ng) / (L / ng) ** 3


def wavenumbers(L: float, ng: int):
    """k of every mode of a real FFT of an ng^3 mesh (the last axis halved)."""
    k = 2.0 * np.pi * np.fft.fftfreq(ng, d=L / ng)
    kz = 2.0 * np.pi * np.fft.rfftfreq(ng, d=L / ng)
    return np.meshgrid(k, k, kz, indexing="ij")


def solve(rho: np.ndarray, L: float, G: float, r_s: float) -> np.ndarray:
    """Steps 2-4 and the inverse transform: acceleration mesh (3, ng, ng, ng)."""
    ng = rho.shape[0]
    d = L / ng
    kx, ky, kz = wavenumbers(L, ng)
    k2 = kx * kx + ky * ky + kz * kz
    sinc = lambda x: np.sinc(x / np.pi)    # sin x / x
    C = (sinc(kx * d / 2) * sinc(ky * d / 2) * sinc(kz * d / 2)) ** 2
    rk = np.fft.rfftn(rho)
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = -4.0 * np.pi * G * rk * np.exp(-k2 * r_s * r_s) / (k2 * C * C)
    phi[0, 0, 0] = 0.0
    nyq = np.pi * ng / L                   # |k| of the Nyquist plane
    acc = []
    for ka in (kx, ky, kz):
        kd = np.where(np.isclose(np.abs(ka), nyq), 0.0, ka)
        acc.append(np.fft.irfftn(-1j * kd * phi, s=rho.shape, axes=(0, 1, 2)))
    return np.stack(acc)


def interpolate(acc_mesh: np.ndarray, pos, L: float) -> np.ndarray:
    """Step 5: the mesh field at every particle, shape (N, 3)."""
    ng = acc_mesh.shape[1]
    cells, w = cic_weights(np.asarray(pos, np.float64), L, ng)
    flat = acc_mesh.reshape(3, -1)
    return np.stack([(flat[a][cells] * w).sum(1) for a in range(3)], 1)


def accelerations(pos, mass, L: float, ng: int, G: float, r_s: float) -> np.ndarray:
    """Long-range acceleration of every particle, shape (N, 3)."""
    return interpolate(solve(deposit(pos, mass, L, ng), L, G, r_s), pos, L)
