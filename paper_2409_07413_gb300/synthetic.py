"""Seeded synthetic diffraction patterns shaped like single-shot XFEL CDI data.

This module is shared by the tests, the benchmark and the smoke check for BOTH the CUDA
path and the FP64 oracle.  It holds no arithmetic of the reconstruction method itself:
it only draws objects, forms their far-field intensities with numpy's FFT, adds Poisson
noise, and builds the detector masks and the initial support that a user would supply.

All Fourier-space arrays returned here are detector-centred (zero frequency at
``(n//2, n//2)``), as a detector delivers them; real-space arrays (object, support) have
the object near the centre.

Workload recipes (sizes from the paper's data: pnCCD / Jungfrau single shots binned to
N_p = 512 or 256, Sec. "Computational cost and performance"):

* ``pattern_sphere``: a uniform sphere (diameter 20 px) plus two small spheres
  (diameter 4-8 px) at seeded offsets, central beamstop disc r = 3 px.
* ``pattern_ellipsoids``: a union of 3-6 ellipsoid projections inside a given extent,
  density uniform in [0.5, 1] per ellipsoid, central beamstop/hole of radius r, an
  optional horizontal detector gap of ``gap_rows`` rows through the centre, and
  saturation: pixels above the 99.9th percentile clipped and masked.

Photon totals are applied before Poisson noise.  The initial support is the threshold
``|F^-1[Xi I]| >= 0.04 max`` of the masked autocorrelation (centred).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Pattern:
    intensities: np.ndarray  # float32, n x n, detector-centred
    mask: np.ndarray         # uint8, n x n, detector-centred, 1 = measured
    support0: np.ndarray     # uint8, n x n, real space
    truth: np.ndarray        # complex128, n x n, the object (real space)
    n: int
    saturated: np.ndarray | None = None  # uint8, n x n, detector-centred, 1 = saturated (masked)


def _sphere_thickness(n, cy, cx, radius):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    d2 = (y - cy) ** 2 + (x - cx) ** 2
    return 2.0 * np.sqrt(np.clip(radius * radius - d2, 0.0, None))


def _ellipsoid_thickness(n, cy, cx, a, b, c, theta):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    u = (x - cx) * np.cos(theta) + (y - cy) * np.sin(theta)
    v = -(x - cx) * np.sin(theta) + (y - cy) * np.cos(theta)
    q = 1.0 - (u / a) ** 2 - (v / b) ** 2
    return 2.0 * c * np.sqrt(np.clip(q, 0.0, None))


def _disc(n, r):
    y, x = np.mgrid[0:n, 0:n]
    return ((y - n // 2) ** 2 + (x - n // 2) ** 2) <= r * r


def _intensity(obj, photons, rng, noise=True):
    I = np.abs(np.fft.fftshift(np.fft.fft2(obj))) ** 2
    I *= photons / I.sum()
    if noise:
        I = rng.poisson(I).astype(np.float64)
    return I


def autocorrelation_support(I, mask, threshold=0.04):
    """Centred support from the masked autocorrelation of the data."""
    Id = np.fft.ifftshift(np.where(mask > 0, I, 0.0))
    ac = np.abs(np.fft.fftshift(np.fft.ifft2(Id)))
    return (ac >= threshold * ac.max()).astype(np.uint8)


def pattern_sphere(seed=0, n=64, photons=1e5, beamstop=3, noise=True):
    rng = np.random.default_rng(seed)
    c = n / 2.0
    obj = _sphere_thickness(n, c, c, 10.0)
    for _ in range(2):
        d = rng.uniform(4.0, 8.0)
        ang = rng.uniform(0, 2 * np.pi)
        rr = rng.uniform(6.0, 12.0)
        obj = obj + _sphere_thickness(n, c + rr * np.sin(ang), c + rr * np.cos(ang), d / 2)
    I = _intensity(obj, photons, rng, noise)
    mask = np.ones((n, n), np.uint8)
    if beamstop > 0:
        mask[_disc(n, beamstop)] = 0
    S0 = autocorrelation_support(I, mask)
    return Pattern(I.astype(np.float32), mask, S0, obj.astype(np.complex128), n)


def pattern_ellipsoids(seed=0, n=512, extent=120.0, photons=1e7, beamstop=12, gap_rows=20,
                       saturate=True, noise=True):
    rng = np.random.default_rng(seed)
    c = n / 2.0
    obj = np.zeros((n, n))
    for _ in range(int(rng.integers(3, 7))):
        a = rng.uniform(0.12, 0.3) * extent
        b = rng.uniform(0.12, 0.3) * extent
        cz = rng.uniform(0.12, 0.3) * extent
        lim = extent / 2 - max(a, b)
        cy = c + rng.uniform(-lim, lim)
        cx = c + rng.uniform(-lim, lim)
        rho = rng.uniform(0.5, 1.0)
        obj = obj + rho * _ellipsoid_thickness(n, cy, cx, a, b, cz, rng.uniform(0, np.pi))
    I = _intensity(obj, photons, rng, noise)
    mask = np.ones((n, n), np.uint8)
    if beamstop > 0:
        mask[_disc(n, beamstop)] = 0
    if gap_rows > 0:
        mask[n // 2 - gap_rows // 2: n // 2 - gap_rows // 2 + gap_rows, :] = 0
    sat = np.zeros((n, n), bool)
    if saturate:
        lim = np.percentile(I[mask > 0], 99.9)
        sat = (I > lim) & (mask > 0)
        I = np.where(sat, lim, I)
        mask[sat] = 0
    I = np.where(mask > 0, I, 0.0)
    S0 = autocorrelation_support(I, mask)
    return Pattern(I.astype(np.float32), mask, S0, obj.astype(np.complex128), n, sat.astype(np.uint8))


def config_pattern(name: str, seed: int = 0) -> Pattern:
    """Synthetic pattern for a named workload.

    ``sphere64``   64x64, 1e5 photons, beamstop r=3.
    ``ell512``     512x512, 120 px extent, 1e7 photons, beamstop r=12, 20-row gap,
                   99.9th-percentile saturation.
    ``ell1024``    1024x1024, 200 px extent, 1e8 photons, hole r=24, 30-row gap (a split
                   two-panel detector; no saturation).
    ``ellN``       any other supported N (96 ... 768): extent 0.25 N, photons log-uniform in
                   [1e6, 1e7], beamstop r = N/40, gap N/25 rows.
    """
    if name == "sphere64":
        return pattern_sphere(seed)
    if name == "ell512":
        return pattern_ellipsoids(seed, 512, 120.0, 1e7, 12, 20, True)
    if name == "ell1024":
        return pattern_ellipsoids(seed, 1024, 200.0, 1e8, 24, 30, False)
    if name.startswith("ell"):
        n = int(name[3:])
        rng = np.random.default_rng(10_000 + seed)
        photons = float(10 ** rng.uniform(6, 7))
        return pattern_ellipsoids(seed, n, 0.25 * n, photons, max(2, n // 40), max(2, n // 25), True)
    raise ValueError(name)


def noise_free_object(seed=0, n=32, size=8):
    """A real positive object in a small box (oversampling >= 2 per axis), with its exact
    support; intensities unmasked and noise-free.  For recovery tests."""
    rng = np.random.default_rng(seed)
    obj = np.zeros((n, n))
    o = (n - size) // 2
    obj[o:o + size, o:o + size] = rng.uniform(0.2, 1.0, (size, size))
    S = (obj > 0).astype(np.uint8)
    # orthonormal transform, so that the object is an exact fixed point of a unitary P_M
    I = np.abs(np.fft.fftshift(np.fft.fft2(obj, norm="ortho"))) ** 2
    return Pattern(I.astype(np.float64), np.ones((n, n), np.uint8), S, obj.astype(np.complex128), n)


def population_state(seed, batch, n, support_frac=0.25):
    """Random complex population state and supports for operator-level tests."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    S = (rng.random((batch, n, n)) < support_frac).astype(np.uint8)
    return x, S


def random_modulus(seed, n, masked_frac=0.1):
    """Random positive modulus in DFT order and a random mask (operator-level tests)."""
    rng = np.random.default_rng(seed + 1)
    M = rng.uniform(0.1, 2.0, (n, n))
    mask = (rng.random((n, n)) >= masked_frac).astype(np.uint8)
    return M, mask


def poisson_arrivals(seed, rate_hz, duration_s):
    """Seeded Poisson arrival times (a hit stream), in seconds."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.asarray(out)
        out.append(t)
