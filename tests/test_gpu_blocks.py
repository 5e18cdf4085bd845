"""Position-blocked LSQML (the residuals of B positions resident at a time,
for scans whose residuals exceed device memory) against the FP64 oracle and
against the resident run.  Same arithmetic; only the grouping of the sums
changes, so results agree with the resident run to FP32 rounding and with
the oracle to the usual 1e-4."""
import numpy as np
import pytest

from gpu_cases import illuminated, scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api
from util import align_global, rel_l2

pytestmark = pytest.mark.gpu


def _run(c, n, **kw):
    with api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], **kw) as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(c["O0"], c["P0"])
        r.iterate("lsqml", n)
        return r.get_object(), r.get_probe(), r.fourier_error()


CASES = [(32, 1, 1, 1), (32, 1, 4, 4), (32, 3, 4, 7), (64, 1, 2, 5), (96, 1, 2, 8), (16, 2, 1, 3)]


@pytest.mark.parametrize("M,K,C,B", CASES, ids=lambda v: str(v))
def test_blocked_lsqml_parity(M, K, C, B):
    c = scan(M, K, grid=3, photons=1e6, mask_frac=0.02)
    n = 6
    Ob, Pb, Eb = _run(c, n, cluster=C, block_positions=B)
    Or, Pr, Er = _run(c, n, cluster=C)
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], n)
    m = illuminated(c["P"], c["pos"], c["shape"])
    assert rel_l2(align_global(Ob, Oc, m), Oc, m) < 1e-4 and rel_l2(Pb, Pc) < 1e-4
    assert rel_l2(Ob, Or, m) < 1e-5 and rel_l2(Pb, Pr) < 1e-5
    assert abs(Eb - Er) <= 1e-5 * Er


@pytest.mark.parametrize("opts", [dict(likelihood="poisson"), dict(probe_ortho=1), dict(probe_start=3),
                                  dict(istore="bf16")], ids=str)
def test_blocked_lsqml_options(opts):
    c = scan(32, 3, grid=3, photons=1e5)
    Ob, Pb, _ = _run(c, 5, cluster=4, block_positions=4, **opts)
    Or, Pr, _ = _run(c, 5, cluster=4, **opts)
    m = illuminated(c["P"], c["pos"], c["shape"])
    assert rel_l2(Ob, Or, m) < 1e-5 and rel_l2(Pb, Pr) < 1e-5


def test_blocked_step_equals_whole_and_one_block_is_resident():
    c = scan(32, 1, grid=3, photons=1e5)
    with api.Reconstruction(32, 1, 9, c["shape"], block_positions=4) as a:
        a.set_data(c["I"].astype(np.float32), c["pos"])
        a.set_init(c["O0"], c["P0"])
        a.iterate("lsqml", 3)
        Oa, Pa = a.get_object(), a.get_probe()
    with api.Reconstruction(32, 1, 9, c["shape"], block_positions=4) as b:
        b.set_data(c["I"].astype(np.float32), c["pos"])
        b.set_init(c["O0"], c["P0"])
        for _ in range(3):
            b.iterate("lsqml", 1)
        assert np.array_equal(Oa, b.get_object()) and np.array_equal(Pa, b.get_probe())
    # B >= J is the resident path, bit for bit
    O9, P9, _ = _run(c, 3, block_positions=9)
    O0, P0, _ = _run(c, 3)
    assert np.array_equal(O9, O0) and np.array_equal(P9, P0)


def test_blocked_rejects_dm_and_subpixel():
    c = scan(32, 1, grid=2)
    with api.Reconstruction(32, 1, len(c["pos"]), c["shape"], block_positions=2) as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        with pytest.raises(api.PtychoError) as e:
            r.iterate("dm", 1)
        assert e.value.name == "UNSUPPORTED"
        r.iterate("epie", 1)   # ePIE holds no residual array
        r.iterate("lsqml", 1)
    with pytest.raises(api.PtychoError) as e:
        api.Reconstruction(32, 1, 4, (64, 64), block_positions=2, subpixel=8)
    assert e.value.name == "UNSUPPORTED"
    with pytest.raises(api.PtychoError) as e:
        api.Reconstruction(32, 1, 4, (64, 64), block_positions=-1)
    assert e.value.name == "ARG"


def test_blocked_batch_member():
    """A blocked member inside a batch's captured graph equals the same
    member run alone, bit for bit."""
    cases = [scan(32, 1, grid=3, photons=1e5, seed=41), scan(64, 1, grid=3, photons=1e5, seed=42)]
    opts = [dict(block_positions=4), dict()]
    members = [dict(M=c["M"], K=c["K"], J=len(c["pos"]), obj_shape=c["shape"], **o) for c, o in zip(cases, opts)]
    with api.Batch(members) as b:
        for m, c in zip(b.members, cases):
            m.set_data(c["I"].astype(np.float32), c["pos"])
            m.set_init(c["O0"], c["P0"])
        b.iterate("lsqml", 3)
        got = [(m.get_object(), m.get_probe()) for m in b.members]
    for (Og, Pg), c, o in zip(got, cases, opts):
        Os, Ps, _ = _run(c, 3, **o)
        assert np.array_equal(Og, Os) and np.array_equal(Pg, Ps)
