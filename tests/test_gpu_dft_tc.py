"""The tensor-core DFT engine (fft_engine = PTYCHO_DFT_TENSOR_BF16X3, 64^2
detector, one mode) against the FP64 oracle.

Tolerances.  Each 1-D transform is one product with the DFT matrix in BF16
with a three-term split: the dropped lo*lo term and the rounding of the lo
parts leave about 2^-17 relative error per product, accumulated in FP32 over
the 128 real terms of a row; a Fourier pass chains four such transforms and
the residual is a difference of two nearly equal far fields, so single passes
are held to 1e-4 (against 2e-5 for the FP32 FFT) and the Fourier error to
2e-5.  Reconstructions: O and P after 1 and 10 iterations to the FP32 path's
1e-4 (measured: 3e-6 and 7e-5 for LSQML).  DM's exit waves take every pass's
transform error directly (psi += F^-1 (Pi(Z) - Z)): about 2.5e-5 per
iteration, so they are held to 5e-4 after 10 iterations (measured 2.4e-4)."""
import numpy as np
import pytest

from gpu_cases import illuminated, scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api
from util import align_global, rel_l2

pytestmark = pytest.mark.gpu

ENG = "tensor_bf16x3"
TOL_TC_PASS = 1e-4
TOL_TC_E = 2e-5
TOL_REC = 1e-4
TOL_TC_PSI = 5e-4


def _recon(c, **kw):
    r = api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], fft_engine=ENG, **kw)
    r.set_data(c["I"].astype(np.float32), c["pos"])
    r.set_init(c["O0"], c["P0"])
    return r


def test_forward_model():
    c = scan(64, 1, grid=3)
    with api.Reconstruction(64, 1, len(c["pos"]), c["shape"], fft_engine=ENG) as r:
        r.set_positions(c["pos"])
        r.set_init(c["O"], c["P"])
        I = r.simulate()
    assert rel_l2(I, c["I"]) < TOL_TC_PASS


@pytest.mark.parametrize("istore", ["f32", "f16", "bf16"])
def test_residual_and_error(istore):
    c = scan(64, 1, grid=3, photons=1e6, mask_frac=0.05)
    pos_i = orc.round_positions(c["pos"])
    with _recon(c, istore=istore) as r:
        chi = r.fourier_residual()
        E = r.fourier_error()
    with api.Reconstruction(64, 1, len(c["pos"]), c["shape"], istore=istore) as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(c["O0"], c["P0"])
        chi32, E32 = r.fourier_residual(), r.fourier_error()
    # against the FFT path with the same amplitude storage: the transform's own error
    assert rel_l2(chi, chi32) < TOL_TC_PASS
    assert abs(E - E32) <= TOL_TC_E * E32
    if istore == "f32":
        assert rel_l2(chi, orc.fourier_residual(c["O0"], c["P0"], pos_i, c["I"])) < TOL_TC_PASS
        E_ref = orc.fourier_error(c["O0"], c["P0"], pos_i, c["I"])
        assert abs(E - E_ref) <= TOL_TC_E * E_ref


@pytest.mark.parametrize("alg,n", [("dm", 1), ("dm", 10), ("lsqml", 1), ("lsqml", 10)])
def test_algorithm_parity(alg, n):
    c = scan(64, 1, grid=3, photons=1e6, mask_frac=0.02)
    with _recon(c) as r:
        r.iterate(alg, n)
        Og, Pg, E = r.get_object(), r.get_probe(), r.fourier_error()
        psi = r.get_exit_waves() if alg == "dm" else None
    Oc, Pc, psic = orc.reconstruct(alg, c["O0"], c["P0"], c["pos"], c["I"], n)
    m = illuminated(c["P"], c["pos"], c["shape"])
    assert rel_l2(align_global(Og, Oc, m), Oc, m) < TOL_REC
    assert rel_l2(Pg, Pc) < TOL_REC
    E_own = orc.fourier_error(Og.astype(np.complex128), Pg.astype(np.complex128), orc.round_positions(c["pos"]), c["I"])
    assert abs(E - E_own) <= TOL_TC_E * E_own
    if psi is not None:
        assert rel_l2(psi, psic) < (TOL_REC if n == 1 else TOL_TC_PSI)


def test_poisson_and_subpixel_run_on_the_engine():
    """Poisson-likelihood residuals and sub-pixel probe tables go through the
    same kernel (the mode's detector factor; the position's probe bin)."""
    c = scan(64, 1, grid=3, photons=1e5)
    pos_i = orc.round_positions(c["pos"])
    with _recon(c, likelihood="poisson") as r:
        chi = r.fourier_residual()
    ref = orc.fourier_residual(c["O0"], c["P0"], pos_i, c["I"], likelihood="poisson")
    assert rel_l2(chi, ref) < TOL_TC_PASS
    from gpu_cases import subpixel_scan
    s = subpixel_scan(64, 1, 8, grid=3)
    with api.Reconstruction(64, 1, len(s["pos"]), s["shape"], fft_engine=ENG, subpixel=8) as r:
        r.set_positions(s["pos"])
        r.set_init(s["O"], s["P"])
        I = r.simulate()
    assert rel_l2(I, s["I"]) < TOL_TC_PASS


def test_deterministic_and_step_equals_whole():
    c = scan(64, 1, grid=4, photons=1e5)
    with _recon(c) as a:
        a.iterate("lsqml", 3)
        Oa = a.get_object()
    with _recon(c) as b:
        for _ in range(3):
            b.iterate("lsqml", 1)
            b.get_object()
        Ob = b.get_object()
    assert np.array_equal(Oa, Ob)


def test_unsupported_shape_is_rejected():
    with pytest.raises(api.PtychoError) as e:
        api.Reconstruction(128, 1, 4, (200, 200), fft_engine=ENG)
    assert e.value.name == "UNSUPPORTED"


def test_engine_autotuner_and_auto_engine():
    """ptycho_autotune_engine times both engines where both are compiled and
    keeps the faster; fft_engine = "auto" then builds a context with that
    engine, whose results equal an explicit context of the same engine bit
    for bit.  Elsewhere only the register FFT is compiled and is chosen."""
    eng, C, ms = api.autotune_engine(64, 1)
    assert eng in ("register", "tensor_bf16x3") and C >= 1 and ms > 0
    assert api.autotune_engine(64, 1) == (eng, C, ms)     # cached
    eng128, C128, _ = api.autotune_engine(128, 1)
    assert eng128 == "register" and C128 == api.autotune(128, 1)[0]
    c = scan(64, 1, grid=3, photons=1e5, seed=31)
    outs = []
    for kw in (dict(fft_engine="auto", cluster=-1), dict(fft_engine=eng, cluster=C)):
        with api.Reconstruction(64, 1, len(c["pos"]), c["shape"], **kw) as r:
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(c["O0"], c["P0"])
            r.iterate("lsqml", 2)
            outs.append((r.get_object(), r.get_probe(), r.fourier_error()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]
