"""Small seeded scans for the GPU parity tests (inputs only; the expected
values always come from the FP64 oracle)."""
from __future__ import annotations

import numpy as np

from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import synth

# (M, K, cluster) combinations compiled into the library
COMPILED = [
    (16, 1, 1), (16, 1, 2), (16, 2, 1), (16, 3, 1), (16, 3, 2),
    (32, 1, 1), (32, 1, 2), (32, 1, 4), (32, 2, 2), (32, 3, 1), (32, 3, 4),
    (64, 1, 1), (64, 1, 2), (64, 1, 4), (64, 3, 2), (64, 3, 4),
    (128, 1, 2), (128, 1, 4), (128, 1, 8), (128, 3, 4), (128, 3, 8),
    (256, 1, 4), (256, 1, 8), (256, 1, 16),
    (96, 1, 1), (96, 1, 2), (96, 1, 4), (192, 1, 2), (192, 1, 4), (192, 1, 8),
]


def scan(M, K, grid=3, step=None, jitter=1, seed=0, photons=None, mask_frac=0.0, ragged=True):
    """Truth, intensities (FP64 oracle forward model) and a flat/perturbed start.

    The object is sized so that patches touch its last row/column and its
    shape is not a multiple of the 32x64 object tile (ragged tails)."""
    step = step or max(2, M // 4)
    P = synth.make_probe(M, K, R=M / 4.0, sigma=M / 16.0, c=0.6 / M)
    pos = synth.raster_positions(grid, grid, step, jitter, jitter, seed=seed + 1)
    ny = int(np.rint(pos[:, 0]).max()) + M
    nx = int(np.rint(pos[:, 1]).max()) + M
    if not ragged:
        ny, nx = -(-ny // 16) * 16, -(-nx // 16) * 16
    O = synth.make_object(ny, nx, seed=seed + 2, smooth=max(1.0, M / 16))
    pos_i = orc.round_positions(pos)
    I = orc.far_field_intensity(O, P, pos_i)
    if photons:
        I = synth.poisson(I * photons / I.sum(axis=(1, 2)).mean(), seed=seed + 3)
    if mask_frac > 0:
        rng = np.random.default_rng(seed + 4)
        I = np.where(rng.random(I.shape) < mask_frac, -1.0, I)
    O0 = synth.flat_object(ny, nx)
    P0 = synth.noisy_probe(P, 0.1, seed=seed + 5)
    return dict(M=M, K=K, P=P, O=O, pos=pos, I=I, O0=O0, P0=P0, shape=(ny, nx))


def illuminated(P, pos, shape, frac=0.1):
    den = orc.object_denominator(P, orc.round_positions(pos), shape)
    return den >= frac * den.max()


def subpixel_scan(M, K, S, grid=3, step=None, seed=0, photons=None, mask_frac=0.0):
    """A scan at fractional positions (raster + uniform offsets in [0, 1)),
    float32 like the values the ABI receives, with the oracle's sub-pixel
    forward model at 1/S-pixel quantisation."""
    step = step or max(2, M // 4)
    rng = np.random.default_rng(seed + 30)
    P = synth.make_probe(M, K, R=M / 4.0, sigma=M / 16.0, c=0.6 / M)
    base = synth.raster_positions(grid, grid, step, 1, 1, seed=seed + 1)
    pos = (np.rint(base) + rng.uniform(0.0, 1.0, base.shape)).astype(np.float32).astype(np.float64)
    corner, delta = orc.subpixel_positions(pos, S)
    ny = int(corner[:, 0].max()) + M
    nx = int(corner[:, 1].max()) + M
    O = synth.make_object(ny, nx, seed=seed + 2, smooth=max(1.0, M / 16))
    I = orc.far_field_intensity(O, P, corner, delta)
    if photons:
        I = synth.poisson(I * photons / I.sum(axis=(1, 2)).mean(), seed=seed + 3)
    if mask_frac > 0:
        I = np.where(rng.random(I.shape) < mask_frac, -1.0, I)
    O0 = synth.flat_object(ny, nx)
    P0 = synth.noisy_probe(P, 0.1, seed=seed + 5)
    return dict(M=M, K=K, S=S, P=P, O=O, pos=pos, corner=corner, delta=delta, I=I, O0=O0, P0=P0, shape=(ny, nx))
