"""Soft convergence checks of the oracle (the paper prints no error curve, so
these are sanity checks, not pins): from a flat object and a perturbed probe
the Fourier error of each algorithm falls on noise-free data."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import synth


def _case():
    M, K = 32, 1
    P = synth.make_probe(M, K, R=10.0, sigma=2.0, c=0.04)
    pos = synth.raster_positions(5, 5, 8, 1, 2, seed=4)
    ny, nx = synth.object_shape_for(pos, M, margin=3, multiple=4)
    O = synth.make_object(ny, nx, seed=5)
    pos_i = orc.round_positions(pos)
    I = orc.far_field_intensity(O, P, pos_i)
    return P, O, pos, I, synth.flat_object(ny, nx), synth.noisy_probe(P, 0.05, seed=6)


@pytest.mark.parametrize("alg", ["epie", "dm", "lsqml"])
def test_error_decreases(alg):
    P, O, pos, I, O0, P0 = _case()
    pos_i = orc.round_positions(pos)
    e0 = orc.fourier_error(O0, P0, pos_i, I)
    Oc, Pc, _ = orc.reconstruct(alg, O0, P0, pos, I, 20, seed=3, probe_start=5)
    e1 = orc.fourier_error(Oc, Pc, pos_i, I)
    assert e1 < 0.5 * e0, (alg, e0, e1)
