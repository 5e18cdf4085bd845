"""Comparison helpers shared by the tests (no reconstruction arithmetic)."""
from __future__ import annotations

import numpy as np


def rel_l2(a: np.ndarray, b: np.ndarray, mask: np.ndarray | None = None) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    if mask is not None:
        a = a[mask]
        b = b[mask]
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def align_global(a: np.ndarray, ref: np.ndarray, mask: np.ndarray | None = None) -> np.ndarray:
    """Multiply a by the complex scalar c minimising ||c a - ref|| (global phase and scale)."""
    aa = a[mask] if mask is not None else a.ravel()
    rr = ref[mask] if mask is not None else ref.ravel()
    den = np.vdot(aa, aa)
    c = np.vdot(aa, rr) / den if abs(den) > 0 else 1.0
    return a * c


def small_scan(M=16, K=2, grid=3, step=6, jitter=1, seed=0, margin=2):
    """A tiny scan for CPU pins: probe, object, integer positions."""
    from paper_2202_03144_b300 import synth

    P = synth.make_probe(M, K, R=M / 4.0, sigma=M / 16.0, c=0.3 / M)
    pos = synth.raster_positions(grid, grid, step, jitter, margin + jitter, seed=seed + 7)
    ny, nx = synth.object_shape_for(pos, M, margin=margin + jitter, multiple=4)
    O = synth.make_object(ny, nx, seed=seed + 11, smooth=1.5)
    return P, O, pos
