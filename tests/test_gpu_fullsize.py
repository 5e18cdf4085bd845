"""Parity at the full size of the headline workload, in the launch
configuration bench.py times (256^2 detector, 10,000 positions on a 100 x 100
raster at step 24 px, 2640^2 object, 16-CTA clusters).

The FP64 oracle cannot run 10,000 frames in a test, so:
* sampled outputs it computes one by one: the Fourier residual and the
  forward model of 8 positions spread over the scan (corners, edges, middle);
* properties that hold at any size: whole mode == step mode bit for bit, and
  noise-free data is a fixed point of one LSQML and one DM iteration.
The residual of a position depends only on its own frame: the sampled
positions get noisy frames of the true object from the oracle's forward model,
all others seeded synthetic frames.  The residual is taken at a start whose
far field covers the data's band: where data asks for amplitude and the
model's far field is at rounding-noise level (a flat object under a smooth
probe), the projected phase is noise-determined in FP32 and FP64 alike."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api, synth

pytestmark = pytest.mark.gpu

M, K, G, STEP = 256, 1, 100, 24
SAMPLE = [0, 99, 9900, 9999, 4950, 5049, 1234, 8765]


@pytest.fixture(scope="module")
def workload():
    P = synth.make_probe(M, K, R=80.0, sigma=16.0, c=0.00125)
    pos = synth.raster_positions(G, G, STEP, 2, 2, seed=2000)
    O = synth.make_object(2640, 2640, seed=1000)
    P0 = synth.make_probe(M, K, R=88.0, sigma=16.0, c=0.00125)
    rng = np.random.default_rng(77)
    I = rng.gamma(0.5, 40.0, size=(G * G, M, M)).astype(np.float32)
    Is = orc.far_field_intensity(O, P, orc.round_positions(pos[SAMPLE]))
    I[SAMPLE] = synth.poisson(Is * 1e5 / Is.sum(axis=(1, 2)).mean(), seed=78).astype(np.float32)
    I[:, :3, :3] = -1.0  # a few masked pixels in every frame
    return P, O, pos, P0, I


def test_fullsize_residual_and_forward_sampled(workload):
    torch = pytest.importorskip("torch")
    P, O, pos, P0, I = workload
    J = len(pos)
    # a start whose far field covers the data's band (another random object,
    # the probe with 10% noise), so the projection is well conditioned
    O0 = synth.make_object(2640, 2640, seed=1001)
    P0 = synth.noisy_probe(P, 0.1, seed=79)
    with api.Reconstruction(M, K, J, O.shape) as r:
        assert r.cluster == 16
        r.set_data(I, pos)
        r.set_init(O0, P0)
        chi = torch.empty((J, K, M, M), dtype=torch.complex64, device="cuda")
        r.fourier_residual(chi)
        torch.cuda.synchronize()
        got = chi[SAMPLE].cpu().numpy()
        del chi
        r.set_init(O, P)
        Isim = torch.empty((J, M, M), dtype=torch.float32, device="cuda")
        r.simulate(Isim)
        torch.cuda.synchronize()
        Ig = Isim[SAMPLE].cpu().numpy()
    pi = orc.round_positions(pos[SAMPLE])
    ref = orc.fourier_residual(O0, P0, pi, I[SAMPLE].astype(np.float64))
    for s in range(len(SAMPLE)):
        e = np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s])
        assert e < 2e-5, (SAMPLE[s], e)
    Iref = orc.far_field_intensity(O, P, pi)
    for s in range(len(SAMPLE)):
        e = np.linalg.norm(Ig[s] - Iref[s]) / np.linalg.norm(Iref[s])
        assert e < 2e-5, (SAMPLE[s], e)


def test_fullsize_dm_pass_sampled(workload):
    """The DM pass at the bench's launch shape (one exchange buffer, four CTAs
    per SM), on sampled exit waves.  From psi = P O_j the first iteration's
    overlap updates return O and P unchanged in exact arithmetic (num = den O)
    and within FP32 rounding on the GPU (checked); the pass then forms
    psi + F^-1 Pi(F(2 phi - psi)) - phi with phi = P O_j of the updated O, P.
    The oracle takes that step from the GPU's own updated O and P (so the
    check isolates the pass from the rounding of the sums, which the
    projection amplifies where the far field is weak: from the start O, P
    position 0 differs by 3.3e-5) and the start psi.  Bound 4e-5, twice the
    single pass's: the pass's input 2 phi - psi has up to three times the
    exit wave's magnitude and its output adds phi to the inverse transform,
    two more FP32 roundings of exit-wave size ahead of and behind the
    projection (measured at most 2.04e-5 over the sampled positions)."""
    torch = pytest.importorskip("torch")
    P, O, pos, P0, I = workload
    J = len(pos)
    O0 = synth.make_object(2640, 2640, seed=1002)
    P0 = synth.noisy_probe(P, 0.1, seed=80)
    with api.Reconstruction(M, K, J, O.shape) as r:
        assert r.cluster == 16
        r.set_data(I, pos)
        r.set_init(O0, P0)
        r.iterate("dm", 1)
        psi = torch.empty((J, K, M, M), dtype=torch.complex64, device="cuda")
        r.get_exit_waves(psi)
        torch.cuda.synchronize()
        got = psi[SAMPLE].cpu().numpy()
        O1, P1 = r.get_object(), r.get_probe()
        del psi
    # the start comes back unchanged up to FP32 rounding
    assert np.linalg.norm(O1 - O0) / np.linalg.norm(O0) < 1e-5
    assert np.linalg.norm(P1 - P0) / np.linalg.norm(P0) < 1e-5
    pi = orc.round_positions(pos[SAMPLE])
    psi0 = orc.exit_waves(O0.astype(np.complex128), P0.astype(np.complex128), pi)
    phi = orc.exit_waves(O1.astype(np.complex128), P1.astype(np.complex128), pi)
    ref = psi0 + orc.ifft2(orc.project(orc.fft2(2.0 * phi - psi0), orc.to_fft_order(I[SAMPLE].astype(np.float64)))) - phi
    errs = [float(np.linalg.norm(got[s_] - ref[s_]) / np.linalg.norm(ref[s_])) for s_ in range(len(SAMPLE))]
    print("full-size DM pass, sampled exit waves against the oracle:", max(errs))
    assert max(errs) < 4e-5, list(zip(SAMPLE, errs))


def test_fullsize_step_mode_equals_whole_mode(workload):
    P, O, pos, P0, I = workload
    outs = []
    for steps in ([2], [1, 1]):
        with api.Reconstruction(M, K, len(pos), O.shape) as r:
            r.set_data(I, pos)
            r.set_init(np.ones_like(O), P0)
            for n in steps:
                r.iterate("lsqml", n)
            outs.append((r.get_object(), r.get_probe()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("alg", ["lsqml", "dm"])
def test_fullsize_truth_is_a_fixed_point(workload, alg):
    torch = pytest.importorskip("torch")
    P, O, pos, P0, _ = workload
    J = len(pos)
    with api.Reconstruction(M, K, J, O.shape) as r:
        r.set_positions(pos)
        r.set_init(O, P)
        Isim = torch.empty((J, M, M), dtype=torch.float32, device="cuda")
        r.simulate(Isim)
        torch.cuda.synchronize()
        r.set_data(Isim, pos)
        r.set_init(O, P)
        r.iterate(alg, 1)
        O1, P1 = r.get_object(), r.get_probe()
    assert np.linalg.norm(O1 - O) / np.linalg.norm(O) < 1e-5
    assert np.linalg.norm(P1 - P) / np.linalg.norm(P) < 1e-5


def test_beyond_2_to_31_elements():
    """33,124 positions of a 256^2 detector: the residual array holds
    2.17e9 complex values (> 2^31), so every index past frame 32,768 needs
    64-bit arithmetic.  Forward model and residuals of frames on both sides
    of that boundary against the oracle, and one LSQML and one DM iteration
    that stay finite."""
    torch = pytest.importorskip("torch")
    G = 182
    J = G * G
    assert J * M * M > 2 ** 31
    P = synth.make_probe(M, K, R=80.0, sigma=16.0, c=0.00125)
    pos = synth.raster_positions(G, G, STEP, 2, 2, seed=2001)
    side = -(-(24 * G + 236) // 16) * 16
    O = synth.make_object(side, side, seed=1002)
    sample = [0, 32767, 32768, J - 1]
    with api.Reconstruction(M, K, J, O.shape) as r:
        r.set_positions(pos)
        r.set_init(O, P)
        I = torch.empty((J, M, M), dtype=torch.float32, device="cuda")
        r.simulate(I)
        torch.cuda.synchronize()
        Is = I[sample].cpu().numpy()
        pi = orc.round_positions(pos[sample])
        Iref = orc.far_field_intensity(O, P, pi)
        for s in range(len(sample)):
            assert np.linalg.norm(Is[s] - Iref[s]) / np.linalg.norm(Iref[s]) < 2e-5, sample[s]
        r.set_data(I, pos)
        O0 = synth.make_object(side, side, seed=1003)
        P0 = synth.noisy_probe(P, 0.1, seed=80)
        r.set_init(O0, P0)
        del I
        chi = torch.empty((J, K, M, M), dtype=torch.complex64, device="cuda")
        r.fourier_residual(chi)
        torch.cuda.synchronize()
        got = chi[sample].cpu().numpy()
        del chi
        ref = orc.fourier_residual(O0, P0, pi, Is.astype(np.float64))
        for s in range(len(sample)):
            assert np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s]) < 2e-5, sample[s]
        r.iterate("lsqml", 1)
        assert np.isfinite(r.fourier_error())
        r.iterate("dm", 1)
        assert np.isfinite(r.fourier_error())
        assert np.all(np.isfinite(r.get_object())) and np.all(np.isfinite(r.get_probe()))


def test_fullsize_subpixel(workload):
    """The same workload at fractional positions (1/8-pixel shifts, 64
    shifted probes): sampled residuals and forward model against the oracle,
    noise-free data a fixed point of one LSQML iteration, whole == step mode."""
    torch = pytest.importorskip("torch")
    P, O, _, _, I = workload
    S = 8
    pos = synth.fractional_positions(synth.raster_positions(G, G, STEP, 2, 2, seed=2000), seed=2002)
    corner, delta = orc.subpixel_positions(pos[SAMPLE], S)
    J = len(pos)
    O0 = synth.make_object(2640, 2640, seed=1001)
    P0 = synth.noisy_probe(P, 0.1, seed=79)
    Is = orc.far_field_intensity(O, P, corner, delta)
    I = I.copy()
    I[SAMPLE] = synth.poisson(Is * 1e5 / Is.sum(axis=(1, 2)).mean(), seed=81).astype(np.float32)
    with api.Reconstruction(M, K, J, O.shape, subpixel=S) as r:
        assert r.cluster == 16
        r.set_data(I, pos)
        r.set_init(O0, P0)
        chi = torch.empty((J, K, M, M), dtype=torch.complex64, device="cuda")
        r.fourier_residual(chi)
        torch.cuda.synchronize()
        got = chi[SAMPLE].cpu().numpy()
        del chi
        r.set_init(O, P)
        Isim = torch.empty((J, M, M), dtype=torch.float32, device="cuda")
        r.simulate(Isim)
        torch.cuda.synchronize()
        Ig = Isim[SAMPLE].cpu().numpy()
        r.set_data(Isim, pos)
        del Isim
        r.set_init(O, P)
        r.iterate("lsqml", 1)
        O1, P1 = r.get_object(), r.get_probe()
    ref = orc.fourier_residual(O0, P0, corner, I[SAMPLE].astype(np.float64), delta=delta)
    for s in range(len(SAMPLE)):
        e = np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s])
        assert e < 2e-5, (SAMPLE[s], e)
    for s in range(len(SAMPLE)):
        e = np.linalg.norm(Ig[s] - Is[s]) / np.linalg.norm(Is[s])
        assert e < 2e-5, (SAMPLE[s], e)
    assert np.linalg.norm(O1 - O) / np.linalg.norm(O) < 1e-5
    assert np.linalg.norm(P1 - P) / np.linalg.norm(P) < 1e-5
    outs = []
    for steps in ([2], [1, 1]):
        with api.Reconstruction(M, K, J, O.shape, subpixel=S) as r:
            r.set_data(I, pos)
            r.set_init(np.ones_like(O), P0)
            for n in steps:
                r.iterate("lsqml", n)
            outs.append((r.get_object(), r.get_probe()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_fullsize_position_blocks(workload):
    """The bench scan with the residuals of 2,500 positions resident at a time
    (4 blocks): two LSQML iterations agree with the resident run to the
    parity tolerance (the probe sums over 10,000 positions, regrouped, differ
    by ~2e-5 in FP32), and whole mode equals step mode."""
    P, O, pos, P0, I = workload
    outs = []
    for B, steps in ((0, [2]), (2500, [2]), (2500, [1, 1])):
        with api.Reconstruction(M, K, len(pos), O.shape, block_positions=B) as r:
            r.set_data(I, pos)
            r.set_init(np.ones_like(O), P0)
            for n in steps:
                r.iterate("lsqml", n)
            outs.append((r.get_object(), r.get_probe()))
    (Or, Pr), (Ob, Pb), (Os, Ps) = outs
    assert np.linalg.norm(Ob - Or) / np.linalg.norm(Or) < 1e-4
    assert np.linalg.norm(Pb - Pr) / np.linalg.norm(Pr) < 1e-4
    assert np.array_equal(Ob, Os) and np.array_equal(Pb, Ps)
