"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (FP32 arithmetic vs FP64):
  * single Fourier passes (forward model, residual, Fourier error): relative
    L2 <= 2e-5 -- a radix FFT of length M in FP32 has rms relative error of a
    few 1e-7 * log2(M), the projection adds a few ulps;
  * reconstructions after n iterations from the same start: relative L2 <= 1e-4
    over the illuminated object region (den_O >= 0.1 max) after global
    complex-scalar alignment, and on the probe; Fourier error to 1e-5 relative.
"""
import numpy as np
import pytest

from gpu_cases import COMPILED, illuminated, scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api, synth
from util import align_global, rel_l2

pytestmark = pytest.mark.gpu

TOL_PASS = 2e-5
TOL_REC = 1e-4


def recon(c, cluster=0, **kw):
    r = api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], cluster=cluster, **kw)
    r.set_data(c["I"].astype(np.float32), c["pos"])
    r.set_init(c["O0"], c["P0"])
    return r


@pytest.mark.parametrize("M,K,C", COMPILED, ids=lambda v: str(v))
def test_forward_model(M, K, C):
    c = scan(M, K, grid=2)
    with api.Reconstruction(M, K, len(c["pos"]), c["shape"], cluster=C) as r:
        assert r.cluster == C
        r.set_positions(c["pos"])
        r.set_init(c["O"], c["P"])
        I = r.simulate()
    assert rel_l2(I, c["I"]) < TOL_PASS


@pytest.mark.parametrize("M,K,C", COMPILED, ids=lambda v: str(v))
def test_fourier_residual_and_error(M, K, C):
    c = scan(M, K, grid=2, mask_frac=0.05)
    with recon(c, cluster=C) as r:
        chi = r.fourier_residual()
        E = r.fourier_error()
    pos_i = orc.round_positions(c["pos"])
    chi_ref = orc.fourier_residual(c["O0"], c["P0"], pos_i, c["I"])
    assert rel_l2(chi, chi_ref) < TOL_PASS
    E_ref = orc.fourier_error(c["O0"], c["P0"], pos_i, c["I"])
    assert abs(E - E_ref) <= 1e-5 * E_ref


def _compare(c, alg, n, cluster=0, seed=0, probe_start=0, **kw):
    with recon(c, cluster=cluster, seed=seed, probe_start=probe_start, **kw) as r:
        r.iterate(alg, n)
        Og, Pg = r.get_object(), r.get_probe()
        E = r.fourier_error()
        psi = r.get_exit_waves() if alg == "dm" else None
    Oc, Pc, psic = orc.reconstruct(alg, c["O0"], c["P0"], c["pos"], c["I"], n, seed=seed, probe_start=probe_start,
                                   **{k: v for k, v in kw.items()
                                      if k in ("reg", "epie_alpha", "epie_beta", "lsqml_beta", "likelihood",
                                               "probe_ortho")})
    m = illuminated(c["P"], c["pos"], c["shape"])
    eo = rel_l2(align_global(Og, Oc, m), Oc, m)
    ep = rel_l2(Pg, Pc)
    E_ref = orc.fourier_error(Oc, Pc, orc.round_positions(c["pos"]), c["I"])
    # the oracle's E at the GPU's own (O, P): isolates the error pass
    E_own = orc.fourier_error(Og.astype(np.complex128), Pg.astype(np.complex128), orc.round_positions(c["pos"]), c["I"])
    out = dict(eo=eo, ep=ep, E=E, E_ref=E_ref, E_own=E_own)
    if psi is not None:
        out["epsi"] = rel_l2(psi, psic)
    return out


ALG_CASES = [
    ("dm", 32, 1, 1), ("dm", 32, 3, 4), ("dm", 64, 1, 2), ("dm", 16, 2, 1),
    ("lsqml", 32, 1, 1), ("lsqml", 32, 3, 1), ("lsqml", 64, 1, 4), ("lsqml", 16, 3, 2),
    ("epie", 32, 1, 1), ("epie", 32, 3, 4), ("epie", 64, 1, 2), ("epie", 16, 1, 2),
    ("dm", 96, 1, 2), ("lsqml", 96, 1, 1), ("lsqml", 192, 1, 4),
    ("epie", 128, 3, 0),  # default: ePIE on its widest compiled cluster (16 CTAs)
]


@pytest.mark.parametrize("alg,M,K,C", ALG_CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("n", [1, 10])
def test_algorithm_parity(alg, M, K, C, n):
    if alg == "epie" and n == 10:
        n = 4
    c = scan(M, K, grid=3, photons=1e6, mask_frac=0.02)
    res = _compare(c, alg, n, cluster=C, seed=7 if alg == "epie" else 0)
    assert res["eo"] < TOL_REC, res
    assert res["ep"] < TOL_REC, res
    assert abs(res["E"] - res["E_ref"]) <= 1e-5 * res["E_ref"] + 1e-12, res
    assert abs(res["E"] - res["E_own"]) <= 1e-5 * res["E_own"], res
    if "epsi" in res:
        assert res["epsi"] < TOL_REC, res


@pytest.mark.parametrize("alg,n", [("dm", 1), ("dm", 4), ("lsqml", 1), ("lsqml", 10)])
def test_bench_launch_shape_parity(alg, n):
    """The 256^2 detector with one mode on the 16-CTA cluster: the DM-pass and
    residual-pass kernels the benchmark times (k_fourier3<256, 1, 16, DM|CHI,
    f32>), iterated from a start away from the truth (so the projection and
    the DM epilogue phi + F^-1 (Pi(Z) - Z) do real work), against the oracle
    to the fixed tolerances: O, P and the DM exit waves to 1e-4; the error
    pass (the GPU's E against the oracle's E at the same (O, P)) to 1e-5.
    E at each side's own result differs besides by the first-order
    propagation of their (O, P) difference, 2 rel(A) / sqrt(E) with
    rel(A) <= eo + ep."""
    c = scan(256, 1, grid=4, mask_frac=0.02)
    res = _compare(c, alg, n, cluster=16)
    assert res["eo"] < TOL_REC, res
    assert res["ep"] < TOL_REC, res
    assert abs(res["E"] - res["E_own"]) <= 1e-5 * res["E_own"], res
    tol_E = 1e-5 + 4.0 * max(res["eo"], res["ep"]) / np.sqrt(res["E_ref"])
    assert abs(res["E"] - res["E_ref"]) <= tol_E * res["E_ref"], res
    if "epsi" in res:
        assert res["epsi"] < TOL_REC, res


@pytest.mark.parametrize("alg", ["dm", "lsqml", "epie"])
def test_fixed_probe_then_update(alg):
    c = scan(32, 1, grid=3, photons=1e6)
    res = _compare(c, alg, 4, probe_start=2, seed=3)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC, res


@pytest.mark.parametrize("alg", ["dm", "lsqml", "epie"])
def test_single_position(alg):
    c = scan(32, 1, grid=1)
    res = _compare(c, alg, 3)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC, res


@pytest.mark.parametrize("alg", ["dm", "lsqml", "epie"])
def test_step_mode_equals_whole_mode(alg):
    """iterate(n) == n x iterate(1) with reads in between, bit for bit (Sec. 3.2
    step mode vs whole mode); and two runs are identical (no atomics)."""
    c = scan(32, 3, grid=3, photons=1e5)
    with recon(c, cluster=4, seed=11) as a:
        a.iterate(alg, 4)
        Oa, Pa = a.get_object(), a.get_probe()
    with recon(c, cluster=4, seed=11) as b:
        for _ in range(4):
            b.iterate(alg, 1)
            b.get_object()
            b.get_probe()
        Ob, Pb = b.get_object(), b.get_probe()
        assert b.iteration == 4
    assert np.array_equal(Oa, Ob) and np.array_equal(Pa, Pb)


def test_device_pointers_match_host():
    torch = pytest.importorskip("torch")
    c = scan(32, 1, grid=3)
    with recon(c) as a:
        a.iterate("dm", 2)
        Oa = a.get_object()
    with api.Reconstruction(32, 1, len(c["pos"]), c["shape"]) as b:
        b.set_data(torch.from_numpy(c["I"].astype(np.float32)).cuda(), c["pos"])
        b.set_init(torch.from_numpy(c["O0"].astype(np.complex64)).cuda(),
                   torch.from_numpy(c["P0"].astype(np.complex64)).cuda())
        b.iterate("dm", 2)
        out = torch.empty(c["shape"], dtype=torch.complex64, device="cuda")
        b.get_object(out)
        torch.cuda.synchronize()
        Ob = out.cpu().numpy()
    assert np.array_equal(Oa, Ob)


@pytest.mark.parametrize("istore,tol", [("f16", 2e-3), ("bf16", 2e-2)])
def test_reduced_precision_storage(istore, tol):
    """sqrt(I) stored as 16-bit with a per-frame scale: after 5 LSQML iterations
    the result stays within the storage's own rounding of the FP64 oracle."""
    c = scan(64, 1, grid=3, photons=1e6)
    res32 = _compare(c, "lsqml", 5)
    with recon(c, istore=istore) as r:
        r.iterate("lsqml", 5)
        Og, Pg = r.get_object(), r.get_probe()
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], 5)
    m = illuminated(c["P"], c["pos"], c["shape"])
    e = rel_l2(align_global(Og, Oc, m), Oc, m)
    assert res32["eo"] < e < tol, (e, res32)


def test_error_paths():
    c = scan(32, 1, grid=2)
    with api.Reconstruction(32, 1, len(c["pos"]), c["shape"]) as r:
        with pytest.raises(api.PtychoError) as e:
            r.iterate("dm", 1)
        assert e.value.name == "STATE"
        bad = c["pos"].copy()
        bad[0, 1] = c["shape"][1] - 31
        with pytest.raises(api.PtychoError) as e:
            r.set_data(c["I"].astype(np.float32), bad)
        assert e.value.name == "BOUNDS"
        I = c["I"].astype(np.float32).copy()
        I[1, 3, 3] = np.nan
        with pytest.raises(api.PtychoError) as e:
            r.set_data(I, c["pos"])
        assert e.value.name == "NONFINITE"
        # the context stays usable after errors
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(c["O0"], c["P0"])
        r.iterate("lsqml", 1)
        assert np.isfinite(r.fourier_error())


def test_profile_and_launch_count():
    c = scan(32, 1, grid=3)
    with recon(c) as r:
        n0 = r.launch_count
        r.set_profiling(True)
        r.iterate("lsqml", 2)
        prof = r.get_profile()
        assert r.launch_count > n0
    assert prof["fourier_chi"]["launches"] == 2 and prof["fourier_chi"]["ms"] > 0


def test_precision_report_16bit_storage():
    """Error of each result against the FP64 oracle after 20 LSQML iterations
    (64^2 probe, 36 positions, Poisson 1e6) for FP32, FP16 and BF16 amplitude
    storage.  FP32 stays within the parity tolerance; FP16 and BF16 within
    their storage rounding (2^-11 and 2^-8 relative on sqrt(I))."""
    c = scan(64, 1, grid=6, step=12, photons=1e6)
    n = 20
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], n)
    E_ref = orc.fourier_error(Oc, Pc, orc.round_positions(c["pos"]), c["I"])
    m = illuminated(c["P"], c["pos"], c["shape"])
    report = {}
    for store in ("f32", "f16", "bf16"):
        with recon(c, istore=store) as r:
            r.iterate("lsqml", n)
            Og, Pg = r.get_object(), r.get_probe()
        E = orc.fourier_error(Og, Pg, orc.round_positions(c["pos"]), c["I"])
        report[store] = dict(object=rel_l2(align_global(Og, Oc, m), Oc, m), probe=rel_l2(Pg, Pc),
                             fourier_error=abs(E - E_ref) / E_ref)
    print("precision report (relative to the FP64 oracle):", report)
    assert max(report["f32"].values()) < 1e-4
    assert max(report["f16"].values()) < 5e-3
    assert max(report["bf16"].values()) < 5e-2


@pytest.mark.parametrize("istore", ["f32", "f16", "bf16"])
def test_set_data_paths_agree(istore):
    """Host frames (staged, double-buffered upload), device frames read in
    place with 16-byte loads, and device frames at an address that is only
    4-byte aligned (scalar path) give the same stored amplitudes: identical
    residuals and Fourier errors."""
    torch = pytest.importorskip("torch")
    c = scan(64, 1, grid=4, photons=1e5)
    I = c["I"].astype(np.float32)
    J, M = I.shape[0], I.shape[1]
    flat = torch.empty(I.size + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(I.ravel()).cuda()
    sources = {"host": I, "device": torch.from_numpy(I).cuda(), "device_unaligned": flat[1:].view(J, M, M)}
    assert sources["device_unaligned"].data_ptr() % 16 == 4
    res = {}
    for name, src in sources.items():
        with api.Reconstruction(M, 1, J, c["shape"], istore=istore) as r:
            r.set_data(src, c["pos"])
            r.set_init(c["O0"], c["P0"])
            chi = torch.empty((J, 1, M, M), dtype=torch.complex64, device="cuda")
            r.fourier_residual(chi)
            res[name] = (r.fourier_error(), chi.cpu().numpy())
    for name in ("device", "device_unaligned"):
        assert res[name][0] == res["host"][0]
        assert np.array_equal(res[name][1], res["host"][1])


def test_set_init_rejects_nonfinite_and_keeps_state():
    c = scan(32, 1, grid=2)
    with recon(c) as r:
        O_before, P_before = r.get_object(), r.get_probe()
        O_bad = c["O0"].copy()
        O_bad[3, 4] = np.inf
        with pytest.raises(api.PtychoError) as e:
            r.set_init(O_bad, c["P0"])
        assert e.value.name == "NONFINITE"
        P_bad = c["P0"].copy()
        P_bad[0, 1, 1] = np.nan
        with pytest.raises(api.PtychoError) as e:
            r.set_init(None, P_bad)
        assert e.value.name == "NONFINITE"
        assert np.array_equal(r.get_object(), O_before) and np.array_equal(r.get_probe(), P_before)
        r.iterate("lsqml", 1)
        assert np.isfinite(r.fourier_error())


def test_get_into_caller_buffers():
    """get_object / get_probe into a numpy array, a pinned host tensor and a
    device tensor all return the same values; wrong shapes or dtypes are
    rejected before any copy."""
    torch = pytest.importorskip("torch")
    c = scan(32, 1, grid=2)
    with recon(c) as r:
        r.iterate("lsqml", 1)
        O = r.get_object()
        out_np = np.empty_like(O)
        assert r.get_object(out_np) is out_np and np.array_equal(out_np, O)
        out_pin = torch.empty(O.shape, dtype=torch.complex64).pin_memory()
        r.get_object(out_pin)
        assert np.array_equal(out_pin.numpy(), O)
        out_dev = torch.empty(O.shape, dtype=torch.complex64, device="cuda")
        r.get_object(out_dev)
        assert np.array_equal(out_dev.cpu().numpy(), O)
        P = r.get_probe()
        P_pin = torch.empty(P.shape, dtype=torch.complex64).pin_memory()
        assert np.array_equal(r.get_probe(P_pin).numpy(), P)
        with pytest.raises(ValueError):
            r.get_object(np.empty(O.shape, np.complex128))
        with pytest.raises(ValueError):
            r.get_probe(torch.empty((1, 2, 2), dtype=torch.complex64))


# Poisson-likelihood LSQML: every compiled kernel form (single CTA, the
# asynchronous-transpose cluster kernel, K > 1 through shared memory, mixed radix)
POISSON_CASES = [(32, 1, 1), (64, 1, 4), (32, 3, 4), (128, 3, 8), (96, 1, 2)]


@pytest.mark.parametrize("M,K,C", POISSON_CASES, ids=lambda v: str(v))
def test_poisson_residual_matches_oracle(M, K, C):
    c = scan(M, K, grid=2, photons=1e5, mask_frac=0.05)
    with recon(c, cluster=C, likelihood="poisson") as r:
        chi = r.fourier_residual()
    chi_ref = orc.fourier_residual(c["O0"], c["P0"], orc.round_positions(c["pos"]), c["I"], likelihood="poisson")
    assert rel_l2(chi, chi_ref) < TOL_PASS


def _poisson_sensitivity(c, n):
    """Relative change of the oracle's own result (object, probe) after n
    Poisson LSQML iterations when its starting object is perturbed by 1e-7
    relative noise: how much FP32-sized rounding the method itself amplifies."""
    rng = np.random.default_rng(2024)
    O0p = c["O0"] * (1 + 1e-7 * rng.standard_normal(c["O0"].shape))
    Oa, Pa, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], n, likelihood="poisson")
    Ob, Pb, _ = orc.reconstruct("lsqml", O0p, c["P0"], c["pos"], c["I"], n, likelihood="poisson")
    m = illuminated(c["P"], c["pos"], c["shape"])
    pos_i = orc.round_positions(c["pos"])
    Ea, Eb = orc.fourier_error(Oa, Pa, pos_i, c["I"]), orc.fourier_error(Ob, Pb, pos_i, c["I"])
    return rel_l2(Ob, Oa, m), rel_l2(Pb, Pa), abs(Eb - Ea) / Ea


@pytest.mark.parametrize("M,K,C", POISSON_CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("n", [1, 6])
def test_lsqml_poisson_parity(M, K, C, n):
    """The Poisson factor I / A^2 amplifies rounding where the model's far
    field is much weaker than the counts (early iterations from a flat
    start): the bound is 1e-4 or 20x the oracle's own response to a 1e-7
    perturbation of its start, whichever is larger."""
    c = scan(M, K, grid=3, photons=1e5, mask_frac=0.02)
    res = _compare(c, "lsqml", n, cluster=C, likelihood="poisson")
    so, sp, se = _poisson_sensitivity(c, n)
    assert res["eo"] < max(TOL_REC, 20 * so) and res["ep"] < max(TOL_REC, 20 * sp), (res, so, sp)
    # E = ||A - sqrt I||^2 / ||sqrt I||^2 moves by at most 2 ||dA|| / ||A - sqrt I|| relative, i.e. about
    # 2 (eo + ep) / sqrt(E) for the model changes measured above
    tol_e = max(1e-5, 20 * se, 4 * max(res["eo"], res["ep"]) / np.sqrt(res["E_ref"]))
    assert abs(res["E"] - res["E_ref"]) <= tol_e * res["E_ref"] + 1e-12, (res, se)
    assert abs(res["E"] - res["E_own"]) <= 1e-5 * res["E_own"], res


@pytest.mark.parametrize("istore", ["f16", "bf16"])
def test_lsqml_poisson_16bit_storage(istore):
    """The Poisson residual squares the stored amplitude: 16-bit storage stays
    within twice its amplitude rounding of the FP32 result."""
    c = scan(64, 1, grid=3, photons=1e6)
    outs = {}
    for store in ("f32", istore):
        with recon(c, istore=store, likelihood="poisson") as r:
            r.iterate("lsqml", 4)
            outs[store] = r.get_object()
    m = illuminated(c["P"], c["pos"], c["shape"])
    tol = {"f16": 2e-3, "bf16": 2e-2}[istore]
    assert rel_l2(outs[istore], outs["f32"], m) < tol


def test_lsqml_poisson_step_equals_whole_and_reduces_nll():
    c = scan(64, 1, grid=4, photons=1e4)
    with recon(c, likelihood="poisson") as a:
        a.iterate("lsqml", 5)
        Oa, Pa = a.get_object(), a.get_probe()
    with recon(c, likelihood="poisson") as b:
        for _ in range(5):
            b.iterate("lsqml", 1)
        Ob, Pb = b.get_object(), b.get_probe()
    assert np.array_equal(Oa, Ob) and np.array_equal(Pa, Pb)
    pos_i = orc.round_positions(c["pos"])
    assert orc.poisson_nll(Oa, Pa, pos_i, c["I"]) < orc.poisson_nll(c["O0"], c["P0"], pos_i, c["I"])


def test_bad_likelihood_rejected():
    c = scan(32, 1, grid=2)
    with pytest.raises(api.PtychoError) as e:
        api.Reconstruction(32, 1, len(c["pos"]), c["shape"], likelihood=7)
    assert e.value.name == "ARG"


def _nonorthogonal_modes(P, seed=3):
    rng = np.random.default_rng(seed)
    K = P.shape[0]
    U, _ = np.linalg.qr(rng.standard_normal((K, K)) + 1j * rng.standard_normal((K, K)))
    Pm = orc.mix_modes(P, U)
    Pm[1] = Pm[1] + 0.4 * Pm[0]
    return Pm


@pytest.mark.parametrize("M,K,C", [(32, 3, 4), (128, 3, 8), (32, 2, 2)], ids=lambda v: str(v))
def test_orthogonalize_probe_matches_oracle(M, K, C):
    c = scan(M, K, grid=2)
    Pm = _nonorthogonal_modes(c["P"])
    with api.Reconstruction(M, K, len(c["pos"]), c["shape"], cluster=C) as r:
        r.set_init(c["O"], Pm)
        r.orthogonalize_probe()
        Pg = r.get_probe()
    Pref, _ = orc.orthogonalize_modes(Pm)
    assert rel_l2(Pg, Pref) < TOL_PASS
    G = np.conj(Pg.reshape(K, -1)) @ Pg.reshape(K, -1).T
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-5 * np.abs(G).max()


@pytest.mark.parametrize("alg,M,K,C", [("dm", 32, 3, 4), ("lsqml", 32, 3, 4), ("epie", 32, 3, 4),
                                       ("lsqml", 128, 3, 8), ("dm", 32, 2, 2)], ids=lambda v: str(v))
def test_algorithm_parity_with_probe_orthogonalisation(alg, M, K, C):
    """Every iteration that updates the probe ends with the modes rotated into
    their orthogonal basis (DM: the exit waves too), as in the oracle."""
    c = scan(M, K, grid=3, photons=1e6, mask_frac=0.02)
    c["P0"] = _nonorthogonal_modes(c["P0"])
    res = _compare(c, alg, 4, cluster=C, seed=5 if alg == "epie" else 0, probe_ortho=True, probe_start=1)
    assert res["eo"] < TOL_REC and res["ep"] < TOL_REC, res
    assert abs(res["E"] - res["E_ref"]) <= 1e-5 * res["E_ref"] + 1e-12, res
    if "epsi" in res:
        assert res["epsi"] < TOL_REC, res


@pytest.mark.parametrize("alg", ["dm", "lsqml", "epie"])
def test_checkpoint_resume_is_bit_identical(alg):
    """Four iterations in one context equal two, a checkpoint (object, probe,
    iteration index, DM exit waves), and two more in a fresh context."""
    c = scan(32, 3, grid=3, photons=1e5)
    kw = dict(cluster=4, seed=11, probe_start=1)
    with recon(c, **kw) as a:
        a.iterate(alg, 4)
        Oa, Pa = a.get_object(), a.get_probe()
    with recon(c, **kw) as b:
        b.iterate(alg, 2)
        state = b.checkpoint()
    assert state["iteration"] == 2 and (("exit_waves" in state) == (alg == "dm"))
    with recon(c, **kw) as d:
        d.restore(state)
        assert d.iteration == 2
        d.iterate(alg, 2)
        Od, Pd = d.get_object(), d.get_probe()
    assert np.array_equal(Oa, Od) and np.array_equal(Pa, Pd)


def test_set_exit_waves_rejects_nonfinite():
    c = scan(32, 1, grid=2)
    with recon(c) as r:
        r.iterate("dm", 1)
        psi = r.get_exit_waves()
        bad = psi.copy()
        bad[0, 0, 1, 1] = np.nan
        with pytest.raises(api.PtychoError) as e:
            api._check(r.ctx, api.lib().ptycho_set_exit_waves(r.ctx, bad.ctypes.data, 0))
        assert e.value.name == "NONFINITE"
        assert np.array_equal(r.get_exit_waves(), psi)
        with pytest.raises(api.PtychoError):
            api._check(r.ctx, api.lib().ptycho_set_iteration(r.ctx, -1))


@pytest.mark.parametrize("dtype,rot,device", [("uint16", 0, False), ("uint16", 1, True), ("uint32", 3, False),
                                              ("float32", 2, True)])
def test_set_data_raw_matches_oracle_preprocessing(dtype, rot, device):
    """Raw frames larger than M around an off-centre zero frequency, with
    saturated pixels and sub-threshold noise: the stored data equal those of
    ptycho_set_data on the oracle's preprocessed frames (identical residuals
    and Fourier errors)."""
    torch = pytest.importorskip("torch")
    c = scan(64, 1, grid=3, photons=1e5)
    J, M = len(c["pos"]), 64
    rng = np.random.default_rng(41)
    H, W, cy, cx = 80, 90, 37.0, 44.0
    raw = rng.poisson(2.0, (J, H, W)).astype(np.float64)
    # the scan's frames (detector-centred) placed so that the oracle's crop undoes the placement
    Ic = orc.preprocess_frames(np.pad(c["I"], ((0, 0), (0, H - M), (0, W - M))), (M / 2, M / 2), M)
    assert np.array_equal(Ic, c["I"])
    y0, x0 = int(cy) - M // 2, int(cx) - M // 2
    frames = np.rint(c["I"]) if dtype != "float32" else c["I"]
    raw[:, y0:y0 + M, x0:x0 + M] = np.maximum(frames, 0)
    raw[:, y0 + 5, x0 + 7] = 4095.0  # saturated at 12 bits
    raw = raw.astype(dtype)
    kw = dict(saturation_bits=12, threshold=3.0, rot90=rot)
    Iref = orc.preprocess_frames(raw, (cy, cx), M, **kw).astype(np.float32)
    assert (Iref == -1).sum() >= J and (Iref == 0).sum() > 0
    res = []
    for use_raw in (True, False):
        with api.Reconstruction(M, 1, J, c["shape"]) as r:
            if use_raw:
                src = torch.from_numpy(raw).cuda() if device else raw
                r.set_data_raw(src, c["pos"], (cy, cx), **kw)
            else:
                r.set_data(Iref, c["pos"])
            r.set_init(c["O0"], c["P0"])
            res.append((r.fourier_residual(), r.fourier_error()))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]


def test_set_data_raw_rejects_bad_parameters():
    c = scan(32, 1, grid=2)
    raw = np.zeros((len(c["pos"]), 40, 40), np.uint16)
    with api.Reconstruction(32, 1, len(c["pos"]), c["shape"]) as r:
        for kw in (dict(rot90=4), dict(saturation_bits=25), dict(saturation_bits=-1)):
            with pytest.raises(api.PtychoError) as e:
                r.set_data_raw(raw, c["pos"], (20, 20), **kw)
            assert e.value.name == "ARG"
        with pytest.raises(ValueError):
            r.set_data_raw(raw.astype(np.int8), c["pos"], (20, 20))


@pytest.mark.parametrize("device", [False, True])
def test_set_data_raw_spans_several_chunks(device):
    """600 raw 16-bit frames of a 256^2 detector (the uploads and the
    preprocessing run in chunks of 512 frames): identical stored data to
    ptycho_set_data on the oracle's preprocessed frames, frames on both
    sides of the chunk boundary included."""
    torch = pytest.importorskip("torch")
    M, J, H, W, cy, cx = 256, 600, 270, 262, 131.0, 129.0
    rng = np.random.default_rng(77)
    raw = rng.poisson(5.0, (J, H, W)).astype(np.uint16)
    raw[:, 10, 10] = 65535
    pos = np.stack([rng.integers(0, 60, J), rng.integers(0, 60, J)], axis=1).astype(np.float64)
    shape = (320, 320)
    kw = dict(saturation_bits=16, threshold=2.0, rot90=1)
    Iref = orc.preprocess_frames(raw, (cy, cx), M, **kw).astype(np.float32)
    out = []
    for use_raw in (True, False):
        with api.Reconstruction(M, 1, J, shape) as r:
            if use_raw:
                r.set_data_raw(torch.from_numpy(raw).cuda() if device else raw, pos, (cy, cx), **kw)
            else:
                r.set_data(Iref, pos)
            r.set_init(np.ones(shape, np.complex64), synth.make_probe(M, 1, R=60.0, sigma=10.0, c=0.002))
            chi = torch.empty((J, 1, M, M), dtype=torch.complex64, device="cuda")
            r.fourier_residual(chi)
            torch.cuda.synchronize()
            out.append((r.fourier_error(), chi[[0, 511, 512, 599]].cpu().numpy()))
            del chi
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])


def test_epie_runs_on_the_widest_cluster_by_default():
    c = scan(128, 3, grid=2)
    with api.Reconstruction(128, 3, len(c["pos"]), c["shape"]) as r:
        assert r.cluster == 8 and r.epie_cluster == 16
    with api.Reconstruction(128, 3, len(c["pos"]), c["shape"], cluster=4) as r:
        assert r.cluster == 4 and r.epie_cluster == 4
    # sub-pixel positions: the per-position Fourier pass takes the same cluster
    with api.Reconstruction(128, 3, len(c["pos"]), c["shape"], subpixel=8) as r:
        assert r.cluster == 8 and r.epie_cluster == 16
    with api.Reconstruction(128, 3, len(c["pos"]), c["shape"], cluster=4, subpixel=8) as r:
        assert r.cluster == 4 and r.epie_cluster == 4
