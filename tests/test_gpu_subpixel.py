"""GPU parity of sub-pixel positions (probe translated by the Fourier shift
theorem, positions quantised to 1/S pixel) against the FP64 oracle.

Same tolerances as the integer path: the shifted-probe table adds four
length-M FP32 transforms per probe value (relative error a few 1e-7), well
inside 2e-5 for single passes and 1e-4 for reconstructions."""
import numpy as np
import pytest

from gpu_cases import subpixel_scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api, synth
from util import align_global, rel_l2

pytestmark = pytest.mark.gpu

TOL_PASS = 2e-5
TOL_REC = 1e-4


def _recon(c, cluster=0, **kw):
    r = api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], cluster=cluster, subpixel=c["S"], **kw)
    r.set_data(c["I"].astype(np.float32), c["pos"])
    r.set_init(c["O0"], c["P0"])
    return r


def _illuminated(c, frac=0.1):
    den = orc.object_denominator(c["P"], c["corner"], c["shape"], c["delta"])
    return den >= frac * den.max()


PASS_CASES = [(16, 1, 1, 2), (32, 3, 4, 8), (64, 1, 2, 16), (96, 1, 2, 8), (128, 3, 8, 4), (192, 1, 4, 8),
              (256, 1, 16, 8)]


@pytest.mark.parametrize("M,K,C,S", PASS_CASES, ids=lambda v: str(v))
def test_subpixel_forward_model(M, K, C, S):
    c = subpixel_scan(M, K, S, grid=2)
    with api.Reconstruction(M, K, len(c["pos"]), c["shape"], cluster=C, subpixel=S) as r:
        r.set_positions(c["pos"])
        r.set_init(c["O"], c["P"])
        I = r.simulate()
    assert rel_l2(I, c["I"]) < TOL_PASS


@pytest.mark.parametrize("M,K,C,S", PASS_CASES, ids=lambda v: str(v))
def test_subpixel_residual_and_error(M, K, C, S):
    c = subpixel_scan(M, K, S, grid=2, mask_frac=0.05)
    with _recon(c, cluster=C) as r:
        chi = r.fourier_residual()
        E = r.fourier_error()
    chi_ref = orc.fourier_residual(c["O0"], c["P0"], c["corner"], c["I"], delta=c["delta"])
    assert rel_l2(chi, chi_ref) < TOL_PASS
    E_ref = orc.fourier_error(c["O0"], c["P0"], c["corner"], c["I"], delta=c["delta"])
    assert abs(E - E_ref) <= 1e-5 * E_ref


def _compare(c, alg, n, cluster=0, probe_start=0, seed=0, **kw):
    with _recon(c, cluster=cluster, probe_start=probe_start, seed=seed, **kw) as r:
        r.iterate(alg, n)
        Og, Pg = r.get_object(), r.get_probe()
        E = r.fourier_error()
        psi = r.get_exit_waves() if alg == "dm" else None
    Oc, Pc, psic = orc.reconstruct(alg, c["O0"], c["P0"], c["pos"], c["I"], n, probe_start=probe_start, seed=seed,
                                   subpixel=c["S"], **{k: v for k, v in kw.items() if k in ("likelihood", "probe_ortho")})
    m = _illuminated(c)
    out = dict(eo=rel_l2(align_global(Og, Oc, m), Oc, m), ep=rel_l2(Pg, Pc), E=E,
               E_ref=orc.fourier_error(Oc, Pc, c["corner"], c["I"], delta=c["delta"]),
               E_own=orc.fourier_error(Og.astype(np.complex128), Pg.astype(np.complex128), c["corner"], c["I"],
                                       delta=c["delta"]))
    if psi is not None:
        out["epsi"] = rel_l2(psi, psic)
    return out


ALG_CASES = [
    ("dm", 32, 1, 1, 8), ("dm", 32, 3, 4, 4), ("dm", 16, 2, 1, 2), ("dm", 96, 1, 2, 16),
    ("lsqml", 32, 1, 1, 8), ("lsqml", 32, 3, 4, 16), ("lsqml", 64, 1, 2, 4), ("lsqml", 16, 3, 2, 2),
    ("lsqml", 192, 1, 4, 8), ("lsqml", 256, 1, 8, 8), ("dm", 128, 3, 8, 8),
    ("epie", 32, 1, 1, 8), ("epie", 32, 3, 4, 4), ("epie", 64, 1, 2, 16), ("epie", 96, 1, 2, 8),
    ("epie", 128, 3, 8, 8), ("epie", 16, 2, 1, 2),
]


@pytest.mark.parametrize("alg,M,K,C,S", ALG_CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("n", [1, 8])
def test_subpixel_algorithm_parity(alg, M, K, C, S, n):
    if M >= 128 and n > 1:
        n = 3
    c = subpixel_scan(M, K, S, grid=3, photons=1e6, mask_frac=0.02)
    res = _compare(c, alg, n, cluster=C, seed=7 if alg == "epie" else 0)
    assert res["eo"] < TOL_REC, res
    assert res["ep"] < TOL_REC, res
    # E is evaluated at each side's own (O, P): besides the 1e-5 of one pass it
    # carries their difference, |dE|/E <= 2 |dA|/|A - sqrt I| ~ 2 rel(A)/sqrt(E)
    # with rel(A) <= eo + ep
    tol_E = 1e-5 + 4.0 * max(res["eo"], res["ep"]) / np.sqrt(res["E_ref"])
    assert abs(res["E"] - res["E_ref"]) <= tol_E * res["E_ref"] + 1e-12, res
    # the error pass itself: the oracle's E at the GPU's own (O, P), fixed 1e-5
    assert abs(res["E"] - res["E_own"]) <= 1e-5 * res["E_own"], res
    if "epsi" in res:
        assert res["epsi"] < TOL_REC, res


@pytest.mark.parametrize("alg", ["dm", "lsqml", "epie"])
def test_subpixel_fixed_probe_then_update(alg):
    c = subpixel_scan(32, 2, 8, grid=3, photons=1e6)
    res = _compare(c, alg, 4, probe_start=2)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC, res


def test_subpixel_poisson_and_orthogonalisation():
    c = subpixel_scan(32, 3, 8, grid=3, photons=1e5)
    res = _compare(c, "lsqml", 4, likelihood="poisson", probe_ortho=True)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC, res
    res = _compare(c, "dm", 4, probe_ortho=True)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC and res["epsi"] < TOL_REC, res


@pytest.mark.parametrize("istore", ["f16", "bf16"])
def test_subpixel_16bit_storage(istore):
    """16-bit amplitude storage with sub-pixel positions against the FP64
    oracle: within the storage rounding (2^-11 and 2^-8 relative on sqrt I)."""
    c = subpixel_scan(64, 1, 8, grid=3, photons=1e6)
    n = 3
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], n, subpixel=8)
    with _recon(c, cluster=2, istore=istore) as r:
        r.iterate("lsqml", n)
        Og, Pg = r.get_object(), r.get_probe()
    m = _illuminated(c)
    tol = 5e-3 if istore == "f16" else 5e-2
    assert rel_l2(align_global(Og, Oc, m), Oc, m) < tol and rel_l2(Pg, Pc) < tol


def test_subpixel_fp16_residuals():
    """FP16 residual storage with sub-pixel positions (the probe sums then
    walk the positions in bin order, two pixels per thread): within the
    FP16-residual bound of the integer path (1e-3) of the oracle, and
    n x iterate(1) == iterate(n) bit for bit."""
    c = subpixel_scan(64, 1, 8, grid=3, photons=1e6)
    n = 3
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], n, subpixel=8)
    with _recon(c, cluster=2, residual_store="f16") as r:
        r.iterate("lsqml", n)
        Og, Pg = r.get_object(), r.get_probe()
    with _recon(c, cluster=2, residual_store="f16") as r:
        for _ in range(n):
            r.iterate("lsqml", 1)
        Os, Ps = r.get_object(), r.get_probe()
    assert np.array_equal(Og, Os) and np.array_equal(Pg, Ps)
    m = _illuminated(c)
    eo, ep = rel_l2(align_global(Og, Oc, m), Oc, m), rel_l2(Pg, Pc)
    print(f"sub-pixel, FP16 residuals: object {eo:.2e} probe {ep:.2e}")
    assert eo < 1e-3 and ep < 1e-3, (eo, ep)


@pytest.mark.parametrize("alg", ["dm", "lsqml"])
def test_subpixel_step_mode_equals_whole_mode(alg):
    c = subpixel_scan(32, 3, 8, grid=3, photons=1e5)
    with _recon(c, cluster=4) as a:
        a.iterate(alg, 4)
        Oa, Pa = a.get_object(), a.get_probe()
    with _recon(c, cluster=4) as b:
        for _ in range(4):
            b.iterate(alg, 1)
            b.get_object()
        Ob, Pb = b.get_object(), b.get_probe()
    assert np.array_equal(Oa, Ob) and np.array_equal(Pa, Pb)


def test_subpixel_integral_positions_match_integer_path():
    """Positions on whole pixels: every shift is zero and the sub-pixel path
    equals the integer one up to the rounding of the zero shift's transforms."""
    c = subpixel_scan(32, 1, 8, grid=3, photons=1e6)
    pos = np.rint(c["pos"])
    corner, delta = orc.subpixel_positions(pos, 8)
    assert not delta.any()
    I = orc.far_field_intensity(c["O"], c["P"], corner).astype(np.float32)
    out = []
    for S in (0, 8):
        with api.Reconstruction(32, 1, len(pos), c["shape"], subpixel=S) as r:
            r.set_data(I, pos)
            r.set_init(c["O0"], c["P0"])
            r.iterate("lsqml", 5)
            out.append((r.get_object(), r.get_probe()))
    assert rel_l2(out[1][0], out[0][0]) < 1e-5 and rel_l2(out[1][1], out[0][1]) < 1e-5


def test_subpixel_epie_step_equals_whole_and_bad_params():
    """Sub-pixel ePIE: n sweeps in one call equal n calls of one sweep, bit for
    bit (the order depends on the iteration index), and the probe is
    orthogonalised after each sweep when asked."""
    c = subpixel_scan(32, 3, 8, grid=3, photons=1e5)
    with _recon(c, cluster=4, seed=5) as a:
        a.iterate("epie", 3)
        Oa, Pa = a.get_object(), a.get_probe()
    with _recon(c, cluster=4, seed=5) as b:
        for _ in range(3):
            b.iterate("epie", 1)
        assert np.array_equal(Oa, b.get_object()) and np.array_equal(Pa, b.get_probe())
    res = _compare(c, "epie", 2, cluster=4, seed=5, probe_ortho=True)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC, res
    for S in (1, 3, 6, 32, -2):
        with pytest.raises(api.PtychoError) as e:
            api.Reconstruction(32, 1, 4, (64, 64), subpixel=S)
        assert e.value.name == "ARG"


def test_subpixel_bounds():
    """The corner of a position within 1/(2S) of the object's edge rounds up
    and the patch falls outside: PTYCHO_ERR_BOUNDS, as for integer positions."""
    M = 32
    with api.Reconstruction(M, 1, 2, (64, 64), subpixel=8) as r:
        r.set_positions(np.array([[0.0, 0.0], [32.0, 31.9]], np.float32))  # 31.9 -> corner 32: fits
        with pytest.raises(api.PtychoError) as e:
            r.set_positions(np.array([[0.0, 0.0], [32.5, 0.0]], np.float32))  # corner 33
        assert e.value.name == "BOUNDS"
        with pytest.raises(api.PtychoError) as e:
            r.set_positions(np.array([[-0.6, 0.0], [0.0, 0.0]], np.float32))  # corner -1
        assert e.value.name == "BOUNDS"


def test_subpixel_dm_converges():
    """The difference map with sub-pixel positions (the probe solved by
    conjugate gradients) lowers the Fourier error over 14 iterations on a scan
    where a diagonal probe update diverges; the oracle agrees at the end."""
    c = subpixel_scan(96, 1, 8, grid=3, photons=1e6, mask_frac=0.02)
    Es = []
    with _recon(c, cluster=2) as r:
        for _ in range(14):
            r.iterate("dm", 1)
            Es.append(r.fourier_error())
        Og, Pg = r.get_object(), r.get_probe()
    assert Es[-1] < 0.01 and Es[-1] < Es[2], Es
    Oc, Pc, _ = orc.reconstruct("dm", c["O0"], c["P0"], c["pos"], c["I"], 14, subpixel=8)
    m = _illuminated(c)
    assert rel_l2(align_global(Og, Oc, m), Oc, m) < TOL_REC and rel_l2(Pg, Pc) < TOL_REC


@pytest.mark.parametrize("M,K,C,S", [(32, 1, 1, 8), (32, 3, 4, 16), (64, 1, 2, 8), (256, 1, 16, 8)],
                         ids=lambda v: str(v))
def test_position_refinement_parity(M, K, C, S):
    """One refinement call against the oracle's: the same fresh residual, the
    per-position 2x2 fit, clipping and step, to 1e-4 pixel (float32
    positions of a few hundred pixels carry ~3e-5)."""
    c = subpixel_scan(M, K, S, grid=3, photons=1e6)
    rng = np.random.default_rng(5)
    start = (c["pos"] + rng.uniform(-0.4, 0.4, c["pos"].shape)).astype(np.float32).astype(np.float64)
    start = np.clip(start, 0.0, np.array(c["shape"]) - c["M"] - 0.5)
    with api.Reconstruction(M, K, len(start), c["shape"], cluster=C, subpixel=S) as r:
        r.set_data(c["I"].astype(np.float32), start)
        r.set_init(c["O"], c["P0"])
        assert np.array_equal(r.get_positions(), start.astype(np.float32))
        r.refine_positions(step=0.8, max_shift=0.3)
        got = r.get_positions().astype(np.float64)
        r.iterate("lsqml", 1)   # the context runs on at the new positions
    ref = orc.refine_positions(c["O"], c["P0"], start, c["I"], S, step=0.8, max_shift=0.3)
    assert np.abs(got - ref).max() < 1e-4, np.abs(got - ref).max()
    assert np.abs(got - start).max() <= 0.8 * 0.3 + 1e-4


def test_position_refinement_recovers_positions():
    """From the true object and probe, repeated refinement walks positions
    perturbed by up to 0.4 px back towards the truth, as the oracle does."""
    c = subpixel_scan(64, 1, 16, grid=4, step=12)
    rng = np.random.default_rng(6)
    start = (c["pos"] + rng.uniform(-0.4, 0.4, c["pos"].shape)).astype(np.float32).astype(np.float64)
    start = np.clip(start, 0.0, np.array(c["shape"]) - c["M"] - 0.5)
    errs = []
    with api.Reconstruction(64, 1, len(start), c["shape"], subpixel=16) as r:
        r.set_data(c["I"].astype(np.float32), start)
        r.set_init(c["O"], c["P"])
        for _ in range(6):
            errs.append(float(np.sqrt(np.mean((r.get_positions() - c["pos"]) ** 2))))
            r.refine_positions()
        errs.append(float(np.sqrt(np.mean((r.get_positions() - c["pos"]) ** 2))))
    assert errs[-1] < 0.5 * errs[0], errs
    assert all(b < a + 1e-3 for a, b in zip(errs, errs[1:])), errs


def test_position_refinement_errors():
    c = subpixel_scan(32, 1, 8, grid=2)
    with api.Reconstruction(32, 1, len(c["pos"]), c["shape"]) as r:   # integer positions
        r.set_data(c["I"].astype(np.float32), c["pos"])
        with pytest.raises(api.PtychoError) as e:
            r.refine_positions()
        assert e.value.name == "UNSUPPORTED"
    with api.Reconstruction(32, 1, len(c["pos"]), c["shape"], subpixel=8) as r:
        with pytest.raises(api.PtychoError) as e:
            r.refine_positions()
        assert e.value.name == "STATE"
        r.set_data(c["I"].astype(np.float32), c["pos"])
        with pytest.raises(api.PtychoError) as e:
            r.refine_positions(step=float("nan"))
        assert e.value.name == "ARG"
        with pytest.raises(api.PtychoError) as e:
            r.refine_positions(max_shift=-1.0)
        assert e.value.name == "ARG"
        before = r.get_positions()
        # a step so large that a patch leaves the object: nothing moves
        r.set_init(c["O"], c["P0"])
        with pytest.raises(api.PtychoError) as e:
            r.refine_positions(step=1e6, max_shift=1e3)
        assert e.value.name == "BOUNDS"
        assert np.array_equal(r.get_positions(), before)
        r.iterate("lsqml", 1)


def test_subpixel_checkpoint_with_refined_positions():
    """A run that refines positions, checkpointed and resumed in a new
    context (data set with the original positions), ends bit for bit where
    the uninterrupted run ends."""
    c = subpixel_scan(32, 1, 8, grid=3, photons=1e6)

    def fresh():
        r = _recon(c, cluster=1)
        return r

    with fresh() as a:
        a.iterate("lsqml", 2)
        a.refine_positions(step=0.7)
        a.iterate("lsqml", 2)
        state = a.checkpoint()
        a.refine_positions(step=0.7)
        a.iterate("lsqml", 2)
        Oa, Pa, pa = a.get_object(), a.get_probe(), a.get_positions()
    with fresh() as b:
        b.restore(state)
        assert np.array_equal(b.get_positions(), state["positions"])
        b.refine_positions(step=0.7)
        b.iterate("lsqml", 2)
        assert np.array_equal(b.get_object(), Oa) and np.array_equal(b.get_probe(), Pa)
        assert np.array_equal(b.get_positions(), pa)


@pytest.mark.parametrize("alg", ["dm", "lsqml", "epie"])
def test_subpixel_edge_cases(alg):
    """One position; every position in the same bin (one probe-sum bin holds
    them all, the other bins are empty); positions exactly on half pixels
    (the corner rounds up, the shift is -1/2)."""
    from paper_2202_03144_b300 import synth
    M, S = 32, 8
    P = synth_probe(M)
    O = synth.make_object(72, 72, seed=3, smooth=2.0)
    # a random start: from a flat one, with so few positions, the oracle
    # itself moves its probe by ~3e-3 when the start is perturbed by 1e-7
    O0 = synth.make_object(72, 72, seed=4, smooth=2.0)
    P0 = synth.noisy_probe(P, 0.1, seed=5)
    cases = [np.array([[5.3, 7.8]]),
             np.array([[4.25, 6.25], [9.25, 14.25], [20.25, 3.25], [30.25, 30.25]]),
             np.array([[4.5, 6.5], [9.5, 14.5], [20.5, 3.5]])]
    for raw in cases:
        raw = raw.astype(np.float32).astype(np.float64)
        corner, delta = orc.subpixel_positions(raw, S)
        I = orc.far_field_intensity(O, P, corner, delta)
        with api.Reconstruction(M, 1, len(raw), O.shape, subpixel=S) as r:
            r.set_data(I.astype(np.float32), raw)
            r.set_init(O0, P0)
            r.iterate(alg, 3)
            Og, Pg = r.get_object(), r.get_probe()
        Oc, Pc, _ = orc.reconstruct(alg, O0, P0, raw, I, 3, subpixel=S)
        den = orc.object_denominator(P, corner, O.shape, delta)
        m = den >= 0.1 * den.max()
        assert rel_l2(align_global(Og, Oc, m), Oc, m) < TOL_REC and rel_l2(Pg, Pc) < TOL_REC, raw


def synth_probe(M):
    from paper_2202_03144_b300 import synth
    return synth.make_probe(M, 1, R=M / 4.0, sigma=M / 16.0, c=0.6 / M)


def test_refinement_improves_reconstruction():
    """LSQML from positions perturbed by up to 0.5 px, refining them after
    every iteration, ends with a lower Fourier error and positions closer to
    the truth (up to their common shift) than the same run without
    refinement (an end-to-end check of the feature; the parity of one
    refinement step is tested above)."""
    from paper_2202_03144_b300 import synth
    c = subpixel_scan(64, 1, 16, grid=5, step=12, photons=1e6)
    rng = np.random.default_rng(12)
    start = (c["pos"] + rng.uniform(-0.5, 0.5, c["pos"].shape)).astype(np.float32).astype(np.float64)
    start = np.clip(start, 0.0, np.array(c["shape"]) - c["M"] - 0.5)
    O0 = synth.make_object(*c["shape"], seed=77, smooth=2.0)
    out = {}
    for refine in (False, True):
        with api.Reconstruction(64, 1, len(start), c["shape"], subpixel=16) as r:
            r.set_data(c["I"].astype(np.float32), start)
            r.set_init(O0, c["P0"])
            for _ in range(30):
                r.iterate("lsqml", 1)
                if refine:
                    r.refine_positions(step=1.0, max_shift=0.25)
            err = r.get_positions() - c["pos"]
            err = err - err.mean(axis=0)   # a common shift of all positions is not observable
            out[refine] = (r.fourier_error(), float(np.sqrt(np.mean(err ** 2))))
    (E0, d0), (E1, d1) = out[False], out[True]
    assert E1 < 0.8 * E0 and d1 < d0, out


def _offset_scan(M, K, S, offsets, grid=3, seed=40):
    """A raster whose positions carry the given fractional offsets (cycled
    over the positions in scan order), with the oracle's sub-pixel forward
    model."""
    step = max(2, M // 4)
    P = synth.make_probe(M, K, R=M / 4.0, sigma=M / 16.0, c=0.6 / M)
    base = np.rint(synth.raster_positions(grid, grid, step, 1, 1, seed=seed + 1))
    off = np.array([offsets[i % len(offsets)] for i in range(len(base))], dtype=np.float64)
    pos = (base + off).astype(np.float32).astype(np.float64)
    corner, delta = orc.subpixel_positions(pos, S)
    ny, nx = int(corner[:, 0].max()) + M, int(corner[:, 1].max()) + M
    O = synth.make_object(ny, nx, seed=seed + 2, smooth=max(1.0, M / 16))
    I = orc.far_field_intensity(O, P, corner, delta)
    I = synth.poisson(I * 1e6 / I.sum(axis=(1, 2)).mean(), seed=seed + 3)
    return dict(M=M, K=K, S=S, P=P, O=O, pos=pos, corner=corner, delta=delta, I=I,
                O0=synth.make_object(ny, nx, seed=seed + 4, smooth=max(1.0, M / 16)),
                P0=synth.noisy_probe(P, 0.1, seed=seed + 5), shape=(ny, nx))


@pytest.mark.parametrize("M,K,C", [(32, 3, 4), (128, 3, 8)], ids=lambda v: str(v))
@pytest.mark.parametrize("frames", ["one_bin", "every_position"])
def test_subpixel_epie_frame_paths(M, K, C, frames):
    """The sub-pixel ePIE sweep takes the step's maxima from the frame
    change when the probe's frame moves, else from a separate maxima
    kernel.  One bin for every position (after the first, the frame never
    moves) and alternating bins in visiting order (identity order: it moves
    at every position) each against the oracle, two sweeps."""
    S = 8
    offsets = [(0.3, 0.6)] if frames == "one_bin" else [(0.3, 0.6), (0.8, 0.1)]
    c = _offset_scan(M, K, S, offsets)
    bins = {tuple(b) for b in np.round(c["delta"] * S).astype(int)}
    assert len(bins) == len(offsets)
    res = _compare(c, "epie", 2, cluster=C, seed=0)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC, res


@pytest.mark.parametrize("M,K,C", [(64, 1, 2), (128, 3, 8)], ids=lambda v: str(v))
def test_subpixel_epie_dependent_launch_is_exact(M, K, C):
    """The sweep's per-position kernels are issued with programmatic
    dependent launch; with profiling on (events between launches) they are
    ordinary launches.  Both must give the same bits: every kernel waits for
    its predecessor before touching what it writes or reads."""
    c = subpixel_scan(M, K, 8, grid=4, photons=1e6)
    out = []
    for prof in (False, True):
        with _recon(c, cluster=C, seed=3) as r:
            r.set_profiling(prof)
            r.iterate("epie", 2)
            out.append((r.get_object(), r.get_probe()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
