"""FP16 storage of LSQML's residuals (residual_store = PTYCHO_R_F16): the
residual passes read half the bytes; chi is rounded to FP16 (11 significant
bits) once, when the Fourier pass writes it, and every sum, step size and
update stays FP32 / FP64.

Bounds.  The update is linear in chi: its relative error is that rounding,
2^-12 rms per element (round to nearest), averaged over the overlapping
positions of each pixel -- a few 1e-4 of the update, much less of the
object and probe themselves; over iterations the rounding is re-injected
each time, like the FP16 amplitude storage.  After 1 and 5 iterations the
object and probe stay within 1e-3 of the FP64 oracle (measured in the test
output), and within FP16 storage's own rounding of the FP32-residual run."""
import numpy as np
import pytest

from gpu_cases import illuminated, scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api
from util import align_global, rel_l2

pytestmark = pytest.mark.gpu

TOL_R16 = 1e-3


def _run(c, n, **kw):
    with api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], **kw) as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(c["O0"], c["P0"])
        r.iterate("lsqml", n)
        return r.get_object(), r.get_probe(), r.fourier_error()


@pytest.mark.parametrize("M,K,C", [(64, 1, 1), (256, 1, 16), (128, 3, 8), (32, 3, 4)], ids=str)
@pytest.mark.parametrize("n", [1, 5])
def test_fp16_residuals_against_oracle(M, K, C, n):
    c = scan(M, K, grid=3, photons=1e6, mask_frac=0.02)
    Og, Pg, E = _run(c, n, cluster=C, residual_store="f16")
    O32, P32, E32 = _run(c, n, cluster=C)
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], n)
    m = illuminated(c["P"], c["pos"], c["shape"])
    eo, ep = rel_l2(align_global(Og, Oc, m), Oc, m), rel_l2(Pg, Pc)
    d32 = rel_l2(Og, O32, m)
    print(f"FP16 residuals, M={M} K={K} n={n}: object {eo:.2e} probe {ep:.2e} (FP32 residuals: {d32:.2e} apart)")
    assert eo < TOL_R16 and ep < TOL_R16, (eo, ep)
    assert abs(E - E32) <= 1e-3 * E32


def test_fp16_residuals_deterministic_blocked_and_step_mode():
    """Bit-identical repeat runs, n x iterate(1) == iterate(n), and the
    position-blocked iteration (residuals of B positions at a time) with the
    same FP16 storage.  The blocked sums regroup FP32 additions (~1e-7
    relative); from the second iteration on, chi is computed from objects that
    differ by that much, and wherever an FP32 value straddles an FP16 rounding
    boundary its stored residual moves by a whole FP16 unit (2^-11 relative).
    The two runs therefore agree to the parity bound 1e-4 (measured 1.3e-5
    after 3 iterations), not to the 1e-5 of FP32 residuals."""
    c = scan(64, 1, grid=4, photons=1e5)
    Oa, Pa, _ = _run(c, 3, residual_store="f16")
    Ob, Pb, _ = _run(c, 3, residual_store="f16")
    assert np.array_equal(Oa, Ob) and np.array_equal(Pa, Pb)
    with api.Reconstruction(64, 1, len(c["pos"]), c["shape"], residual_store="f16") as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(c["O0"], c["P0"])
        for _ in range(3):
            r.iterate("lsqml", 1)
            r.get_object()
        Os = r.get_object()
    assert np.array_equal(Oa, Os)
    Ok, Pk, _ = _run(c, 3, residual_store="f16", block_positions=5)
    m = illuminated(c["P"], c["pos"], c["shape"])
    eo, ep = rel_l2(Ok, Oa, m), rel_l2(Pk, Pa)
    print(f"FP16 residuals, blocked against whole: object {eo:.2e} probe {ep:.2e}")
    assert eo < 1e-4 and ep < 1e-4, (eo, ep)


def test_fp16_residuals_leave_dm_and_the_residual_call_fp32():
    """DM's exit waves and ptycho_fourier_residual's output do not take the
    FP16 storage: both equal the FP32 context's results bit for bit."""
    c = scan(64, 1, grid=3, photons=1e5)
    outs = []
    for store in ("f32", "f16"):
        with api.Reconstruction(64, 1, len(c["pos"]), c["shape"], residual_store=store) as r:
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(c["O0"], c["P0"])
            chi = r.fourier_residual()
            r.iterate("dm", 2)
            outs.append((chi, r.get_object(), r.get_exit_waves()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("width", ["even", "odd"])
def test_fp16_residual_probe_sums_any_alignment(width):
    """The probe sums take two adjacent pixels per thread from FP16
    residuals; the object pair is one 16-byte load only where the patch's
    first column and the object's row length are both even, two 8-byte loads
    otherwise.  Positions of both column parities, on objects of even and odd
    width, match the oracle as the other cases do, and the FP32-residual run
    to within the FP16 rounding."""
    c = scan(64, 1, grid=4, photons=1e6)
    ny, nx = c["shape"]
    nx2 = nx + (nx & 1) + (1 if width == "odd" else 0)
    O0 = np.ones((ny, nx2), np.complex128)
    O0[:, :nx] = c["O0"]
    c = dict(c, O0=O0, shape=(ny, nx2))
    cols = orc.round_positions(c["pos"])[:, 1].astype(int)
    assert (cols % 2 == 0).any() and (cols % 2 == 1).any()
    n = 3
    Og, Pg, E = _run(c, n, residual_store="f16")
    O32, P32, E32 = _run(c, n)
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], n)
    m = illuminated(c["P"], c["pos"], c["shape"])
    eo, ep = rel_l2(align_global(Og, Oc, m), Oc, m), rel_l2(Pg, Pc)
    d32 = rel_l2(Pg, P32)
    print(f"FP16 residuals, {width} width: object {eo:.2e} probe {ep:.2e} (probe {d32:.2e} from FP32 residuals)")
    assert eo < TOL_R16 and ep < TOL_R16, (eo, ep)
    assert d32 < TOL_R16 and abs(E - E32) <= 1e-3 * E32
