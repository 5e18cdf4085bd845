"""Seeded synthetic inputs shaped like the scans of a ptychography beamline.

This module only draws inputs: probes, objects, scan positions, initial
guesses and shot noise.  It holds none of the reconstruction arithmetic (no
forward model, no Fourier transform, no update rule), so the FP64 oracle and
the CUDA path can both be fed from it without sharing any of the method.

All generators are deterministic functions of their arguments; every random
draw goes through ``numpy.random.default_rng(seed)`` (PCG64).

Shapes follow the workloads the library is measured on:

* probe: a top-hat of radius ``R`` softened by a Gaussian edge of width
  ``sigma`` with a quadratic (defocus) phase ``c * r**2``; extra incoherent
  modes are the base probe times low-order polynomials, orthonormalised and
  given fixed powers;
* object: a smoothed uniform amplitude in [0.8, 1.0] and a smoothed Gaussian
  phase field in [-pi/2, pi/2];
* positions: a jittered raster or a Fermat spiral, as integer-valued floats
  (y, x) of each patch's top-left corner, optionally with uniform fractional
  offsets (scan steps that are not whole pixels).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage, special

__all__ = [
    "make_probe",
    "make_object",
    "raster_positions",
    "fractional_positions",
    "spiral_positions",
    "object_shape_for",
    "flat_object",
    "noisy_probe",
    "poisson",
    "mode_powers",
    "scan_config",
]


def mode_powers(K: int) -> np.ndarray:
    """Fractional power of each incoherent probe mode (sums to 1)."""
    table = {1: [1.0], 2: [0.8, 0.2], 3: [0.7, 0.2, 0.1], 4: [0.6, 0.2, 0.1, 0.1]}
    if K not in table:
        raise ValueError(f"K={K} modes not supported by the generator")
    return np.asarray(table[K], dtype=np.float64)


def make_probe(M: int, K: int = 1, R: float = 20.0, sigma: float = 4.0,
               c: float = 0.02, total_power: float | None = None) -> np.ndarray:
    """Complex probe modes [K, M, M] (complex128).

    ``total_power`` is sum over modes and pixels of |P|^2; by default the
    base mode keeps its natural amplitude (peak 1) and the modes share that
    power according to :func:`mode_powers`.
    """
    y, x = np.meshgrid(np.arange(M) - M / 2.0, np.arange(M) - M / 2.0, indexing="ij")
    r = np.hypot(y, x)
    amp = 0.5 * special.erfc((r - R) / (math.sqrt(2.0) * sigma))
    base = amp * np.exp(1j * c * r * r)
    shapes = [np.ones_like(r), y / R, x / R, (y / R) * (x / R)][:K]
    modes = []
    for s in shapes:
        v = base * s
        for u in modes:  # Gram-Schmidt against earlier modes
            v = v - np.vdot(u, v) * u
        v = v / np.linalg.norm(v)
        modes.append(v)
    modes = np.stack(modes)
    if total_power is None:
        total_power = float(np.sum(np.abs(base) ** 2))
    w = np.sqrt(mode_powers(K) * total_power)
    return modes * w[:, None, None]


def make_object(ny: int, nx: int, seed: int, smooth: float = 3.0) -> np.ndarray:
    """Complex object [ny, nx] (complex128): amplitude in [0.8, 1], phase in [-pi/2, pi/2]."""
    rng = np.random.default_rng(seed)
    a = ndimage.gaussian_filter(rng.uniform(0.0, 1.0, (ny, nx)), smooth, mode="wrap")
    a = 0.8 + 0.2 * (a - a.min()) / max(a.max() - a.min(), 1e-300)
    ph = ndimage.gaussian_filter(rng.standard_normal((ny, nx)), smooth, mode="wrap")
    ph = -math.pi / 2 + math.pi * (ph - ph.min()) / max(ph.max() - ph.min(), 1e-300)
    return a * np.exp(1j * ph)


def raster_positions(ny: int, nx: int, step: float, jitter: int, offset: float,
                     seed: int) -> np.ndarray:
    """[ny*nx, 2] float64 (y, x) raster with integer jitter uniform in {-jitter..jitter}."""
    rng = np.random.default_rng(seed)
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([iy.ravel() * step, ix.ravel() * step], axis=1) + offset
    if jitter > 0:
        pos = pos + rng.integers(-jitter, jitter + 1, size=pos.shape)
    return pos.astype(np.float64)


def fractional_positions(pos: np.ndarray, seed: int) -> np.ndarray:
    """Whole-pixel positions plus a uniform [0, 1) offset per coordinate (a
    scan whose steps are not whole pixels), as float32 values in float64."""
    rng = np.random.default_rng(seed)
    out = np.rint(pos) + rng.uniform(0.0, 1.0, pos.shape)
    return out.astype(np.float32).astype(np.float64)


def spiral_positions(n: int, spacing: float, center: tuple[float, float]) -> np.ndarray:
    """Fermat spiral r = a*sqrt(i + 1/2), theta = i * golden angle, with the mean
    nearest-neighbour distance equal to ``spacing``; rounded to integers.

    The spiral's geometry scales linearly with a, so a is the spacing over
    the mean nearest-neighbour distance of the a = 1 spiral."""
    from scipy.spatial import cKDTree

    golden = math.radians(137.50776405003785)
    i = np.arange(n, dtype=np.float64)
    r = np.sqrt(i + 0.5)
    t = i * golden
    unit = np.stack([r * np.sin(t), r * np.cos(t)], axis=1)
    if n > 1:
        d, _ = cKDTree(unit).query(unit, k=2)
        a = spacing / float(d[:, 1].mean())
    else:
        a = spacing
    p = unit * a + np.asarray(center, dtype=np.float64)[None, :]
    return np.rint(p)


def object_shape_for(pos: np.ndarray, M: int, margin: int = 8, multiple: int = 16) -> tuple[int, int]:
    """Smallest object (rounded up to ``multiple``) that holds every patch plus a margin."""
    p = np.rint(pos)
    ny = int(p[:, 0].max()) + M + margin
    nx = int(p[:, 1].max()) + M + margin
    ny = -(-ny // multiple) * multiple
    nx = -(-nx // multiple) * multiple
    return ny, nx


def flat_object(ny: int, nx: int) -> np.ndarray:
    return np.ones((ny, nx), dtype=np.complex128)


def noisy_probe(P: np.ndarray, level: float, seed: int) -> np.ndarray:
    """P plus complex Gaussian noise of rms ``level`` times P's rms."""
    rng = np.random.default_rng(seed)
    rms = math.sqrt(float(np.mean(np.abs(P) ** 2)))
    n = rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape)
    return P + level * rms / math.sqrt(2.0) * n


def poisson(I: np.ndarray, seed: int) -> np.ndarray:
    """Shot noise: an independent Poisson draw per pixel (float64 counts)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.maximum(I, 0.0)).astype(np.float64)


def scan_config(name: str, seed: int = 0) -> dict:
    """Probe, object, positions and initial guesses of a named workload.

    ``photons`` is the target mean of the summed frame intensity; the caller
    scales the probe by ``sqrt(photons / mean frame sum)`` after simulating,
    or passes ``total_power``.  Intensities are NOT produced here.
    """
    if name == "dm64":  # 64^2 probe, 256^2 object, 10x10 raster, noise-free
        M, K = 64, 1
        P = make_probe(M, K, R=20.0, sigma=4.0, c=0.02)
        O = make_object(256, 256, seed=1000 + seed)
        pos = raster_positions(10, 10, 16, 2, 24, seed=2000 + seed)
        P0 = noisy_probe(P, 0.05, seed=3000 + seed)
        return dict(M=M, K=K, probe=P, object=O, positions=pos, photons=None,
                    object0=flat_object(256, 256), probe0=P0, noise=False)
    if name == "modes128":  # 128^2 probe, 3 modes, 1024^2 object, 1600-point spiral
        M, K = 128, 3
        # a 1600-point spiral at 20 px mean spacing spans ~940 px: with the
        # 128 px probe the object must be 1088^2 (1024^2 does not hold it)
        P = make_probe(M, K, R=40.0, sigma=8.0, c=0.005)
        pos = spiral_positions(1600, 20.0, (0.0, 0.0))
        pos = pos - pos.min(0) + 8
        ny, nx = object_shape_for(pos, M, margin=8, multiple=16)
        O = make_object(ny, nx, seed=1000 + seed)
        P0 = make_probe(M, K, R=44.0, sigma=8.0, c=0.005)
        return dict(M=M, K=K, probe=P, object=O, positions=pos, photons=1e5,
                    object0=flat_object(ny, nx), probe0=P0, noise=True)
    if name == "det256":  # 256^2 detector, 100x100 raster at step 24, 2640^2 object
        M, K = 256, 1
        P = make_probe(M, K, R=80.0, sigma=16.0, c=0.00125)
        pos = raster_positions(100, 100, 24, 2, 2, seed=2000 + seed)
        O = make_object(2640, 2640, seed=1000 + seed)
        P0 = make_probe(M, K, R=88.0, sigma=16.0, c=0.00125)
        return dict(M=M, K=K, probe=P, object=O, positions=pos, photons=1e5,
                    object0=flat_object(2640, 2640), probe0=P0, noise=True)
    raise ValueError(f"unknown workload {name!r}")


def batch_members(n: int, seed: int = 0, sizes=(64, 96, 128, 192, 256), jmin=100, jmax=4000):
    """Shapes of the batched workload: n scans with probe sizes drawn from
    ``sizes``, position counts uniform in [jmin, jmax], Fermat spirals with
    spacing round(0.15 M), photons per frame log-uniform in [1e4, 1e6].
    Returns a list of dicts (M, J, spacing, photons, positions, obj_shape)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M = int(rng.choice(sizes))
        J = int(rng.integers(jmin, jmax + 1))
        spacing = float(round(0.15 * M))
        pos = spiral_positions(J, spacing, (0.0, 0.0))
        pos = pos - pos.min(0) + 8
        ny, nx = object_shape_for(pos, M, margin=8, multiple=16)
        photons = float(10 ** rng.uniform(4, 6))
        out.append(dict(M=M, J=J, spacing=spacing, photons=photons, positions=pos, obj_shape=(ny, nx)))
    return out
