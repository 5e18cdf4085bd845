"""The log sink (ptycho_set_log): progress reports with the Fourier error
every few iterations, error reports, and iterates unchanged by the reports."""
import numpy as np
import pytest

from gpu_cases import scan
from paper_2202_03144_b300 import api

pytestmark = pytest.mark.gpu


def _rec(c, **kw):
    r = api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], **kw)
    r.set_data(c["I"].astype(np.float32), c["pos"])
    r.set_init(c["O0"], c["P0"])
    return r


@pytest.mark.parametrize("alg", ["lsqml", "dm", "epie"])
def test_progress_reports_leave_the_iterates_unchanged(alg):
    c = scan(64, 1, grid=3, photons=1e5, seed=7)
    with _rec(c) as a, _rec(c) as b:
        a.iterate(alg, 7)
        msgs = []
        b.set_log(lambda level, m: msgs.append((level, m)), error_every=3)
        b.iterate(alg, 2)   # reports after iterations 3 and 6 of the context, and at the end of each call
        b.iterate(alg, 5)
        assert np.array_equal(a.get_object(), b.get_object())
        assert np.array_equal(a.get_probe(), b.get_probe())
        E_end = b.fourier_error()
    its = [int(m.split("iteration ")[1].split(":")[0]) for lv, m in msgs]
    assert all(lv == 1 for lv, _ in msgs)   # PTYCHO_LOG_INFO
    assert its == [2, 3, 6, 7], msgs
    assert all(m.startswith(f"{alg} iteration") for _, m in msgs)
    E_last = float(msgs[-1][1].split("E = ")[1])
    assert abs(E_last - E_end) <= 1e-9 * E_end   # the same error pass, printed to 10 digits


def test_errors_reach_the_sink_and_the_sink_can_be_removed():
    c = scan(32, 1, grid=2, photons=1e5, seed=8)
    with _rec(c) as r:
        msgs = []
        r.set_log(lambda level, m: msgs.append((level, m)))
        with pytest.raises(api.PtychoError):
            r.iterate("lsqml", -1)
        assert msgs and msgs[-1][0] == 0 and "n_iter" in msgs[-1][1]
        r.iterate("lsqml", 2)                 # error_every = 0: no progress reports
        assert len(msgs) == 1
        r.set_log(None)
        with pytest.raises(api.PtychoError):
            r.iterate("lsqml", -1)
        assert len(msgs) == 1
