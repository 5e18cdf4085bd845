"""Host-side checks of the C ABI that need no GPU: the shared library loads,
exports every entry point include/ptycho.h declares, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2202_03144_b300 import api
from paper_2202_03144_b300.build import LIB, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return api.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ptycho.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ptycho_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["ptycho_create", "ptycho_set_data", "ptycho_set_init", "ptycho_iterate", "ptycho_get_object",
              "ptycho_get_probe", "ptycho_fourier_error", "ptycho_destroy", "ptycho_last_error"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(LIB)
    missing = [s for s in declared_symbols() if not hasattr(raw, s)]
    assert not missing, missing


def test_default_params(lib):
    p = api.default_params()
    assert p.reg == pytest.approx(1e-3) and p.lsqml_beta == pytest.approx(0.9)
    assert p.epie_alpha == 1.0 and p.epie_beta == 1.0 and p.istore == 0 and p.seed == 0


@pytest.mark.parametrize("kw,code", [
    (dict(M=0, K=1, J=4, obj_ny=64, obj_nx=64), "ARG"),
    (dict(M=32, K=1, J=0, obj_ny=64, obj_nx=64), "ARG"),
    (dict(M=32, K=1, J=4, obj_ny=16, obj_nx=64), "ARG"),
    (dict(M=32, K=5, J=4, obj_ny=64, obj_nx=64), "UNSUPPORTED"),
    (dict(M=48, K=1, J=4, obj_ny=64, obj_nx=64), "UNSUPPORTED"),
    (dict(M=32, K=1, J=4, obj_ny=64, obj_nx=64, istore=7), "ARG"),
    (dict(M=32, K=1, J=4, obj_ny=64, obj_nx=64, cluster=3), "UNSUPPORTED"),
])
def test_create_rejects_bad_params(lib, kw, code):
    with pytest.raises(api.PtychoError) as e:
        api.create(api.default_params(**kw))
    assert e.value.name == code


def test_null_context_calls_are_safe(lib):
    L = api.lib()
    assert L.ptycho_iterate(None, 1, 1) == -1
    assert L.ptycho_launch_count(None) == -1
    L.ptycho_destroy(None)


def test_to_pixels_listing1():
    """Listing 1 (sim512): lambda = 2.4797e-10 m, z = 1 m, 172 um pixels, 512 px
    detector, 50 nm step, 110 nm beam -> object pixel lambda z / (M dx_d)."""
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "listing1_sim512.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    step_px = api.to_pixels(vals["lambda"], vals["z"], vals["dx_d"], int(vals["size"]), vals["step"])
    beam_px = api.to_pixels(vals["lambda"], vals["z"], vals["dx_d"], int(vals["size"]), vals["beamSize"])
    dx = vals["lambda"] * vals["z"] / (vals["size"] * vals["dx_d"])
    assert dx == pytest.approx(2.8158e-9, rel=1e-4)
    assert step_px == pytest.approx(17.757, rel=1e-4)
    assert beam_px == pytest.approx(39.065, rel=1e-4)


def _noalloc_args(shift_amp=0, shift_obj=0):
    """Host buffers for the allocation-free call (a CPU test never reaches a
    kernel: these calls must fail in the argument checks)."""
    M, K, J, ny, nx = 32, 1, 2, 64, 64
    obj = np.zeros(ny * nx * 2 + 8, np.float32)
    prb = np.zeros(K * M * M * 2 + 8, np.float32)
    amp = np.zeros(J * M * M + 8, np.float32)
    pos = np.zeros((J, 2), np.float32)
    out = ctypes.c_double()
    o = obj.ctypes.data + (-obj.ctypes.data % 16) + shift_obj
    p = prb.ctypes.data + (-prb.ctypes.data % 16)
    a = amp.ctypes.data + (-amp.ctypes.data % 16) + shift_amp
    keep = (obj, prb, amp, pos)
    return keep, (o, ny, nx, p, M, K, pos.ctypes.data, J, a, ctypes.byref(out), None)


@pytest.mark.parametrize("shift_amp,shift_obj,what", [(4, 0, b"16-byte"), (8, 0, b"16-byte"), (0, 4, b"8-byte")])
def test_noalloc_rejects_misaligned_pointers(lib, shift_amp, shift_obj, what):
    """Misaligned amplitude (16-byte bulk reads) or object (8-byte complex
    loads) pointers are argument errors, caught before any device work."""
    keep, args = _noalloc_args(shift_amp, shift_obj)
    assert lib.ptycho_fourier_error_noalloc(*args) == -1
    assert what in lib.ptycho_last_error(None)


def test_error_message_is_per_thread(lib):
    """The context-free error message is kept per thread: a failure on one
    thread does not overwrite another thread's message."""
    import threading

    keep, args = _noalloc_args(4, 0)
    assert lib.ptycho_fourier_error_noalloc(*args) == -1
    seen = {}

    def other():
        k2, a2 = _noalloc_args(0, 4)
        seen["rc"] = lib.ptycho_fourier_error_noalloc(*a2)
        seen["msg"] = lib.ptycho_last_error(None)

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["rc"] == -1 and b"8-byte" in seen["msg"]
    assert b"16-byte" in lib.ptycho_last_error(None)


def test_new_controls_reject_null(lib):
    assert lib.ptycho_set_wait_limit(None, 5) == -1
    assert lib.ptycho_fp32_fma_peak(None, None, None, None) == -1
    assert lib.ptycho_set_log(None, api.LOG_FN(), None, 0) == -1
    assert lib.ptycho_autotune_engine(1, 1, None, None, None) == -1
    assert api.FFT_ENGINE["auto"] == -1 and api.default_params(fft_engine="auto").fft_engine == -1
    p = api.default_params(M=32, K=1, J=4, obj_ny=64, obj_nx=64)
    assert p.mem_limit == 0
    p2 = api.default_params(M=32, K=1, J=4, obj_ny=64, obj_nx=64, mem_limit=1 << 20)
    assert p2.mem_limit == 1 << 20 and p2.block_positions == 0


def test_fft_engine_validated_before_device_work(lib):
    """An unknown engine is an argument error and a shape the tensor-core DFT
    is not compiled for is unsupported, both before any device call."""
    with pytest.raises(api.PtychoError) as e:
        api.create(api.default_params(M=64, K=1, J=4, obj_ny=96, obj_nx=96, fft_engine=7))
    assert e.value.name == "ARG"
    with pytest.raises(api.PtychoError) as e:
        api.create(api.default_params(M=128, K=1, J=4, obj_ny=160, obj_nx=160, fft_engine="tensor_bf16x3"))
    assert e.value.name == "UNSUPPORTED"
    with pytest.raises(api.PtychoError) as e:
        api.create(api.default_params(M=64, K=3, J=4, obj_ny=96, obj_nx=96, fft_engine="tensor_bf16x3"))
    assert e.value.name == "UNSUPPORTED"


def test_residual_store_validated(lib):
    with pytest.raises(api.PtychoError) as e:
        api.create(api.default_params(M=64, K=1, J=4, obj_ny=96, obj_nx=96, residual_store=3))
    assert e.value.name == "ARG"
    assert api.default_params().residual_store == 0
