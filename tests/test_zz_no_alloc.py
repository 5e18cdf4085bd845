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


def test_noalloc_at_its_position_limit_on_16_cta_clusters():
    """16,384 positions (the limit) on the 256^2 detector, whose Fourier
    kernel runs on 16-CTA clusters: the per-CTA error partials fill the whole
    fixed scratch.  Two calls in a row against the regular call on the same
    data (random object, probe and intensities with masked pixels)."""
    torch = pytest.importorskip("torch")
    M, G = 256, 128
    J = G * G
    iy, ix = np.meshgrid(np.arange(G), np.arange(G), indexing="ij")
    pos = (np.stack([iy.ravel(), ix.ravel()], axis=1) * 8.0).astype(np.float32)
    side = 8 * (G - 1) + M
    gen = torch.Generator(device="cuda").manual_seed(16384)
    O = torch.complex(torch.rand((side, side), device="cuda", generator=gen) + 0.5,
                      torch.rand((side, side), device="cuda", generator=gen) - 0.5)
    P = torch.complex(torch.rand((1, M, M), device="cuda", generator=gen),
                      torch.rand((1, M, M), device="cuda", generator=gen) - 0.5) * 0.1
    I = torch.rand((J, M, M), device="cuda", generator=gen) * 100.0
    I[torch.rand((J, M, M), device="cuda", generator=gen) < 0.01] = -1.0   # masked pixels
    with api.Reconstruction(M, 1, J, (side, side)) as r:
        r.set_data(I, pos)
        r.set_init(O, P)
        E_ref = r.fourier_error()
    # the same data as stored amplitudes: sqrt(I) with the zero frequency at (0, 0)
    Ifft = torch.roll(I, shifts=(-(M // 2), -(M // 2)), dims=(1, 2))
    amp = torch.where(Ifft < 0, torch.full_like(Ifft, -1.0), torch.sqrt(torch.clamp(Ifft, min=0.0)))
    del I, Ifft
    torch.cuda.synchronize()
    for _ in range(2):
        E = api.fourier_error_noalloc(O, P, pos, amp)
        assert abs(E - E_ref) <= TOL_E * E_ref, (E, E_ref)


def test_noalloc_rejects_host_pointers_before_any_launch():
    """A host buffer where device memory is expected is an argument error:
    the pointer's memory type is checked before any device work."""
    import ctypes
    torch = pytest.importorskip("torch")
    M, J = 32, 2
    O_host = np.ones((64, 64, 2), np.float32)
    P = torch.ones((1, M, M), dtype=torch.complex64, device="cuda")
    A = torch.ones((J, M, M), dtype=torch.float32, device="cuda")
    pos = np.zeros((J, 2), np.float32)
    out = ctypes.c_double()
    rc = api.lib().ptycho_fourier_error_noalloc(O_host.ctypes.data, 64, 64, torch.view_as_real(P).data_ptr(), M, 1,
                                                pos.ctypes.data, J, A.data_ptr(), ctypes.byref(out), None)
    assert rc == -1 and b"device memory" in api.lib().ptycho_last_error(None)
