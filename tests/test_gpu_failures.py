"""Failure detection without a GPU fault: a bounded device wait made to run
out, a device-memory cap that turns an allocation into PTYCHO_ERR_OOM, and a
non-finite Fourier error reported as PTYCHO_ERR_DIVERGED.  Each failure comes
from a setting or an input of the host; no kernel faults, traps or hangs, and
the context stays usable afterwards."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api
from tests.gpu_cases import illuminated, scan
from tests.util import align_global, rel_l2

pytestmark = pytest.mark.gpu


def test_wait_limit_runs_out_and_context_recovers():
    """With the wait limit at zero every cluster-transpose wait of the Fourier
    pass gives up at once: the kernel flags it, waits (with its fixed bound)
    for the data still on the way into its shared memory, and returns; the
    next read of the flag reports PTYCHO_ERR_TIMEOUT.  Back at the default
    limit the same context reproduces the oracle's iteration."""
    c = scan(64, 1, grid=3)
    J = len(c["pos"])
    I32 = c["I"].astype(np.float32)
    with api.Reconstruction(64, 1, J, c["shape"], cluster=4) as r:
        assert r.cluster == 4  # the cluster kernel with the bounded transposes
        r.set_data(I32, c["pos"])
        r.set_init(c["O0"], c["P0"])
        r.set_wait_limit(0)
        r.iterate("lsqml", 1)
        with pytest.raises(api.PtychoError) as e:
            r.get_object()
        assert e.value.name == "TIMEOUT"
        r.get_object()  # the flag was cleared by the call that reported it
        with pytest.raises(api.PtychoError) as e:
            r.set_wait_limit(-1)
        assert e.value.name == "ARG"
        r.set_wait_limit(1 << 20)
        r.set_init(c["O0"], c["P0"])
        r.iterate("lsqml", 1)
        Og, Pg = r.get_object(), r.get_probe()
    Oc, Pc, _ = orc.reconstruct("lsqml", c["O0"], c["P0"], c["pos"], c["I"], 1)
    m = illuminated(c["P0"], c["pos"], c["shape"])
    assert rel_l2(align_global(Og, Oc, m), Oc, m) < 1e-4
    assert rel_l2(Pg, Pc) < 1e-4


def test_memory_limit_gives_oom_and_context_stays_usable():
    c = scan(64, 1, grid=3)
    J = len(c["pos"])
    I32 = c["I"].astype(np.float32)
    with api.Reconstruction(64, 1, J, c["shape"]) as r:
        r.set_data(I32, c["pos"])
        r.set_init(c["O0"], c["P0"])
        before = r.memory_used
        r.iterate("lsqml", 1)
        after = r.memory_used
        Oref = r.get_object()
    assert 0 < before < after  # the residual buffers come with the first LSQML iteration
    # a cap below what create needs: create fails cleanly
    with pytest.raises(api.PtychoError) as e:
        api.Reconstruction(64, 1, J, c["shape"], mem_limit=4096)
    assert e.value.name == "OOM"
    # a cap between the two: data and start fit, the iteration's buffers do not
    with api.Reconstruction(64, 1, J, c["shape"], mem_limit=(before + after) // 2) as r:
        r.set_data(I32, c["pos"])
        r.set_init(c["O0"], c["P0"])
        assert r.memory_used == before
        with pytest.raises(api.PtychoError) as e:
            r.iterate("lsqml", 1)
        assert e.value.name == "OOM"
        assert r.memory_used <= (before + after) // 2
        # nothing of the failed call was applied; the context still answers
        np.testing.assert_array_equal(r.get_object(), c["O0"].astype(np.complex64))
        assert np.isfinite(r.fourier_error())
    # and a cap that holds everything gives the unlimited result
    with api.Reconstruction(64, 1, J, c["shape"], mem_limit=after) as r:
        r.set_data(I32, c["pos"])
        r.set_init(c["O0"], c["P0"])
        r.iterate("lsqml", 1)
        np.testing.assert_array_equal(r.get_object(), Oref)


def test_non_finite_error_is_diverged():
    """An object so bright that |F(P O)|^2 overflows float32 gives a
    non-finite Fourier error: PTYCHO_ERR_DIVERGED, and the context stays
    usable."""
    c = scan(64, 1, grid=3)
    J = len(c["pos"])
    with api.Reconstruction(64, 1, J, c["shape"]) as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(c["O"] * 1e20, c["P"])
        with pytest.raises(api.PtychoError) as e:
            r.fourier_error()
        assert e.value.name == "DIVERGED"
        r.set_init(c["O"], c["P"])
        assert r.fourier_error() < 1e-8  # noise-free data at the truth
