"""The allocation-free Fourier error (ptycho_fourier_error_noalloc) against the
context-based ptycho_fourier_error.

That entry point serves callers that cannot call cudaMalloc -- hosts that own
all device memory through their own pool, or live loops that cannot take the
synchronisation an allocation may imply.  It keeps its scratch in one fixed
device array inside the library, so two calls in a row must each give the
same E as the regular call, whatever the previous call left in that array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from gpu_cases import scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api

pytestmark = pytest.mark.gpu

TOL_E = 1e-5   # relative, as for the Fourier error in the parity tests


def _regular_E(c):
    with api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"]) as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(c["O0"], c["P0"])
        return r.fourier_error()


def _noalloc_E(c):
    import torch
    amp = np.sqrt(np.maximum(orc.to_fft_order(c["I"]), 0.0))
    amp = np.where(orc.to_fft_order(c["I"]) < 0, -1.0, amp).astype(np.float32)
    O = torch.from_numpy(c["O0"].astype(np.complex64)).cuda()
    P = torch.from_numpy(c["P0"].astype(np.complex64)).cuda()
    A = torch.from_numpy(amp).cuda()
    torch.cuda.synchronize()
    return api.fourier_error_noalloc(O, P, c["pos"], A)


def test_noalloc_matches_regular_on_two_calls_in_a_row():
    pytest.importorskip("torch")
    cases = [scan(64, 1, grid=3, photons=1e5, mask_frac=0.03, seed=1),
             scan(32, 3, grid=2, photons=1e6, seed=2),
             scan(256, 1, grid=2, photons=1e6, seed=3)]   # 16-CTA clusters
    for c in cases:  # consecutive calls, different sizes, shared scratch
        E_ref = _regular_E(c)
        E = _noalloc_E(c)
        assert abs(E - E_ref) <= TOL_E * E_ref, (E, E_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    M, K, J = 32, 1, 20000
    O = torch.ones((64, 64), dtype=torch.complex64, device="cuda")
    P = torch.ones((K, M, M), dtype=torch.complex64, device="cuda")
    A = torch.ones((1, M, M), dtype=torch.float32, device="cuda")
    pos = np.zeros((J, 2), np.float32)
    with pytest.raises(api.PtychoError) as e:
        api.fourier_error_noalloc(O, P, pos, A)
    assert e.value.name == "ARG" and "16384" in str(e.value)
