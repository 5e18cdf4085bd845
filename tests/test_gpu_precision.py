"""Precision report (the reduced-precision storage and split-precision
tensor-core DFT against the FP64 oracle): 200 LSQML iterations from a random
object and the noisy true probe, on cuts small enough for the oracle to run
whole, with the benchmark's probe, step and photon count.

  * 256^2 detector, 6 x 6 positions: FP32, FP16 and BF16 amplitude storage
    (FP32 transforms);
  * 64^2 detector, 10 x 10 positions: the same three storages with the FP32
    FFT, and FP32 / FP16 storage with the BF16 three-term tensor-core DFT.

Reported per result: relative L2 error of the object (illuminated region,
after global-phase alignment), of the probe, and relative error of the
Fourier error E at the final (O, P).  FP32 stays within the parity
tolerance (1e-4) after 200 iterations.  The reduced-precision variants are
reports, not parity claims: each iteration re-injects the storage's or the
transform's rounding (FP16 sqrt(I): 11 bits, BF16: 8 bits, the split DFT:
about 17 bits per transform) and the iterations carry it forward, growing
roughly linearly with the iteration count.  Measured on a B300 (object /
probe / E):
  256^2: f16 6.2e-3 / 4.1e-3 / 6.1e-4, bf16 1.1e-2 / 6.9e-3 / 5.5e-4;
  64^2:  f16 2.1e-2 / 2.9e-2 / 7.6e-3, bf16 3.6e-2 / 1.1e-1 / 5.1e-3,
         split DFT with FP32 storage 3.9e-3 / 3.4e-3 / 2.0e-3, with FP16
         storage 3.2e-2 / 6.3e-2 / 4.4e-3.
Their bounds are regression guards at about three times those values."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api, synth
from util import align_global, rel_l2

pytestmark = pytest.mark.gpu

N_ITER = 200
BOUND = {"f32": 1e-4, "f16": 0.1, "bf16": 0.35, "tensor_bf16x3/f32": 1.5e-2, "tensor_bf16x3/f16": 0.2}


def _cut(M, G):
    step = 24 * M // 256
    P = synth.make_probe(M, 1, R=80.0 * M / 256, sigma=M / 16.0, c=0.00125 * (256.0 / M) ** 2)
    pos = synth.raster_positions(G, G, step, 2, 2, seed=2000)
    side = -(-(step * (G - 1) + 4 + M) // 16) * 16
    O = synth.make_object(side, side, seed=1000)
    pi = orc.round_positions(pos)
    I = orc.far_field_intensity(O, P, pi)
    sc = 1e5 / I.sum(axis=(1, 2)).mean()
    I = synth.poisson(I * sc, seed=3)
    O0 = synth.make_object(side, side, seed=1001)
    P0 = synth.noisy_probe(P * np.sqrt(sc), 0.1, seed=4)
    den = orc.object_denominator(P, pi, O.shape)
    return dict(M=M, P=P, pos=pos, pi=pi, I=I, O0=O0, P0=P0, mask=den >= 0.1 * den.max(), shape=O.shape)


def _report(c, runs):
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], N_ITER)
    E_ref = orc.fourier_error(Oc, Pc, c["pi"], c["I"])
    out = {}
    for name, kw in runs:
        with api.Reconstruction(c["M"], 1, len(c["pos"]), c["shape"], **kw) as r:
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(c["O0"], c["P0"])
            r.iterate("lsqml", N_ITER)
            Og, Pg = r.get_object(), r.get_probe()
        E = orc.fourier_error(Og.astype(np.complex128), Pg.astype(np.complex128), c["pi"], c["I"])
        out[name] = dict(object=rel_l2(align_global(Og, Oc, c["mask"]), Oc, c["mask"]), probe=rel_l2(Pg, Pc),
                         fourier_error=abs(E - E_ref) / E_ref)
    return out


def test_precision_report_256_detector():
    c = _cut(256, 6)
    rep = _report(c, [(s, dict(istore=s)) for s in ("f32", "f16", "bf16")])
    print(f"precision report, 256^2, 6x6 positions, {N_ITER} LSQML iterations, relative to the FP64 oracle:", rep)
    for name, r in rep.items():
        assert max(r.values()) < BOUND[name], (name, r)


def test_precision_report_64_detector_with_tensor_dft():
    c = _cut(64, 10)
    runs = [(s, dict(istore=s)) for s in ("f32", "f16", "bf16")]
    runs += [(f"tensor_bf16x3/{s}", dict(istore=s, fft_engine="tensor_bf16x3")) for s in ("f32", "f16")]
    rep = _report(c, runs)
    print(f"precision report, 64^2, 10x10 positions, {N_ITER} LSQML iterations, relative to the FP64 oracle:", rep)
    for name, r in rep.items():
        assert max(r.values()) < BOUND[name], (name, r)
