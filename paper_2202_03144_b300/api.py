"""Python binding of the C ABI in include/ptycho.h (ctypes).

Argument marshalling only: every function forwards to the entry point of the
same name in ``libptycho.so``; all computation runs in that library's CUDA
kernels.  Host arrays are numpy; device arrays are torch CUDA tensors (torch is
used for device memory and streams only).  There is no CPU fallback: if the
library is missing or no GPU is present, calls fail with an exception.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

EPIE, DM, LSQML = 0, 1, 2
ALGS = {"epie": EPIE, "dm": DM, "lsqml": LSQML}
I_F32, I_F16, I_BF16 = 0, 1, 2
ISTORE = {"f32": I_F32, "f16": I_F16, "bf16": I_BF16}
LIKELIHOOD = {"amplitude": 0, "poisson": 1}  # PTYCHO_LIK_AMPLITUDE, PTYCHO_LIK_POISSON
FFT_ENGINE = {"auto": -1, "register": 0, "tensor_bf16x3": 1}  # PTYCHO_FFT_AUTO, _REGISTER, PTYCHO_DFT_TENSOR_BF16X3
RESIDUAL_STORE = {"f32": 0, "f16": 1}  # PTYCHO_R_F32, PTYCHO_R_F16

ERRORS = {
    -1: "ARG", -2: "BOUNDS", -3: "NONFINITE", -4: "OOM", -5: "CUDA", -6: "TIMEOUT",
    -7: "DIVERGED", -8: "STATE", -9: "UNSUPPORTED",
}


class PtychoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"PTYCHO_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Params(C.Structure):
    _fields_ = [
        ("M", C.c_int), ("K", C.c_int), ("J", C.c_int), ("obj_ny", C.c_int), ("obj_nx", C.c_int),
        ("istore", C.c_int), ("probe_start", C.c_int),
        ("epie_alpha", C.c_double), ("epie_beta", C.c_double), ("lsqml_beta", C.c_double),
        ("reg", C.c_double), ("seed", C.c_ulonglong), ("stream", C.c_void_p), ("cluster", C.c_int),
        ("likelihood", C.c_int), ("probe_ortho", C.c_int), ("subpixel", C.c_int),
        ("block_positions", C.c_int), ("mem_limit", C.c_ulonglong), ("fft_engine", C.c_int),
        ("residual_store", C.c_int),
    ]


RAW_DTYPES = {"uint16": 0, "uint32": 1, "float32": 2}  # PTYCHO_RAW_U16 / _U32 / _F32


class Preprocess(C.Structure):
    _fields_ = [
        ("raw_h", C.c_int), ("raw_w", C.c_int), ("dtype", C.c_int), ("center_y", C.c_float),
        ("center_x", C.c_float), ("saturation_bits", C.c_int), ("threshold", C.c_float), ("rot90", C.c_int),
    ]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_longlong), ("ms", C.c_double), ("bytes", C.c_double)]


LOG_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_char_p)  # ptycho_log_fn


_lib = None


def lib() -> C.CDLL:
    """Load libptycho.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            from .build import build
            build()
        L = C.CDLL(LIB)
        vp, i, f, d = C.c_void_p, C.c_int, C.c_void_p, C.c_double
        sig = {
            "ptycho_default_params": (None, [C.POINTER(Params)]),
            "ptycho_create": (i, [C.POINTER(vp), C.POINTER(Params)]),
            "ptycho_set_data": (i, [vp, f, f, i]),
            "ptycho_set_positions": (i, [vp, f]),
            "ptycho_set_init": (i, [vp, f, f, i]),
            "ptycho_iterate": (i, [vp, i, i]),
            "ptycho_get_object": (i, [vp, f, i]),
            "ptycho_get_probe": (i, [vp, f, i]),
            "ptycho_get_exit_waves": (i, [vp, f, i]),
            "ptycho_fourier_error": (i, [vp, C.POINTER(d)]),
            "ptycho_simulate": (i, [vp, f, i]),
            "ptycho_fourier_residual": (i, [vp, f, i]),
            "ptycho_iteration": (C.c_longlong, [vp]),
            "ptycho_launch_count": (C.c_longlong, [vp]),
            "ptycho_memory_used": (C.c_longlong, [vp]),
            "ptycho_set_profiling": (i, [vp, i]),
            "ptycho_get_profile": (i, [vp, C.POINTER(KernelStat), i, C.POINTER(i)]),
            "ptycho_cluster_size": (i, [vp]),
            "ptycho_last_error": (C.c_char_p, [vp]),
            "ptycho_fourier_error_noalloc": (i, [f, i, i, f, i, i, f, i, f, C.POINTER(d), vp]),
            "ptycho_set_likelihood": (i, [vp, i]),
            "ptycho_set_wait_limit": (i, [vp, C.c_longlong]),
            "ptycho_set_log": (i, [vp, LOG_FN, vp, i]),
            "ptycho_fp32_fma_peak": (i, [C.POINTER(d), C.POINTER(d), C.POINTER(i), vp]),
            "ptycho_orthogonalize_probe": (i, [vp]),
            "ptycho_set_iteration": (i, [vp, C.c_longlong]),
            "ptycho_epie_cluster_size": (i, [vp]),
            "ptycho_set_data_raw": (i, [vp, vp, C.POINTER(Preprocess), vp, i]),
            "ptycho_set_exit_waves": (i, [vp, vp, i]),
            "ptycho_refine_positions": (i, [vp, d, d]),
            "ptycho_get_positions": (i, [vp, f]),
            "ptycho_batch_create": (i, [C.POINTER(vp), i, C.POINTER(Params), vp]),
            "ptycho_batch_member": (vp, [vp, i]),
            "ptycho_batch_size": (i, [vp]),
            "ptycho_batch_iterate": (i, [vp, i, i]),
            "ptycho_batch_kernels_per_iteration": (C.c_longlong, [vp]),
            "ptycho_batch_set_group_bytes": (i, [vp, C.c_longlong]),
            "ptycho_batch_groups": (i, [vp, C.POINTER(C.c_int)]),
            "ptycho_batch_autotune": (i, [vp, i, i, C.POINTER(C.c_longlong), C.POINTER(i), C.POINTER(d)]),
            "ptycho_batch_set_lanes": (i, [vp, i]),
            "ptycho_batch_lanes": (i, [vp]),
            "ptycho_batch_synchronize": (i, [vp]),
            "ptycho_batch_last_error": (C.c_char_p, [vp]),
            "ptycho_batch_destroy": (None, [vp]),
            "ptycho_autotune": (i, [i, i, C.POINTER(i), C.POINTER(d)]),
            "ptycho_autotune_engine": (i, [i, i, C.POINTER(i), C.POINTER(i), C.POINTER(d)]),
            "ptycho_net_create": (i, [C.POINTER(vp), C.c_ulonglong, i, i, vp]),
            "ptycho_net_num_params": (C.c_longlong, [vp]),
            "ptycho_net_get_params": (i, [vp, f]),
            "ptycho_net_set_params": (i, [vp, f]),
            "ptycho_net_predict": (i, [vp, f, i, f]),
            "ptycho_net_gradients": (i, [vp, f, f, i, f, C.POINTER(d)]),
            "ptycho_net_train_step": (i, [vp, f, f, i, C.c_float, C.POINTER(d)]),
            "ptycho_net_last_error": (C.c_char_p, [vp]),
            "ptycho_net_destroy": (None, [vp]),
            "ptycho_object_patches": (i, [vp, f]),
            "ptycho_warm_start": (i, [vp, vp]),
            "ptycho_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, rc: int) -> None:
    if rc != 0:
        msg = lib().ptycho_last_error(ctx)
        raise PtychoError(rc, msg.decode() if msg else "")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr_in(x, dtype=np.float32):
    """(pointer, on_device, keepalive) of an input array; complex arrays are
    passed as interleaved float32 pairs."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        import torch
        if x.is_complex():
            x = torch.view_as_real(x.to(torch.complex64).contiguous())
        x = x.to(torch.float32).contiguous()
        if not x.is_cuda:
            x = x.numpy()
        else:
            return x.data_ptr(), 1, x
    a = np.asarray(x)
    if np.iscomplexobj(a):
        a = np.ascontiguousarray(a, dtype=np.complex64).view(np.float32)
    else:
        a = np.ascontiguousarray(a, dtype=dtype)
    return a.ctypes.data, 0, a


# ------------------------------------------------------------------ the ABI

def default_params(**kw) -> Params:
    p = Params()
    lib().ptycho_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "istore" and isinstance(v, str):
            v = ISTORE[v]
        if k == "likelihood" and isinstance(v, str):
            v = LIKELIHOOD[v]
        if k == "fft_engine" and isinstance(v, str):
            v = FFT_ENGINE[v]
        if k == "residual_store" and isinstance(v, str):
            v = RESIDUAL_STORE[v]
        if k == "probe_ortho":
            v = int(bool(v))
        setattr(p, k, v)
    return p


def create(params: Params) -> C.c_void_p:
    h = C.c_void_p()
    rc = lib().ptycho_create(C.byref(h), C.byref(params))
    _check(None, rc)
    return h


def set_data(ctx, intensities, positions) -> None:
    ip, dev, keep_i = _ptr_in(intensities)
    pp, _, keep_p = _ptr_in(np.asarray(positions, dtype=np.float32))
    _check(ctx, lib().ptycho_set_data(ctx, ip, pp, dev))


def set_positions(ctx, positions) -> None:
    pp, _, keep = _ptr_in(np.asarray(positions, dtype=np.float32))
    _check(ctx, lib().ptycho_set_positions(ctx, pp))


def set_init(ctx, object=None, probe=None) -> None:
    op, od, ko = _ptr_in(object)
    pp, pd, kp = _ptr_in(probe)
    if object is not None and probe is not None and od != pd:
        set_init(ctx, object, None)
        set_init(ctx, None, probe)
        return
    _check(ctx, lib().ptycho_set_init(ctx, op, pp, od or pd))


def iterate(ctx, alg, n_iter: int) -> None:
    a = ALGS[alg] if isinstance(alg, str) else int(alg)
    _check(ctx, lib().ptycho_iterate(ctx, a, int(n_iter)))


def _get(fn, ctx, shape, out=None):
    """Copy a result into ``out`` (a complex64 torch tensor on the GPU or the
    host -- pinned host memory copies fastest -- or a numpy array), or into a
    new numpy array."""
    if out is not None and _is_torch(out):
        import torch
        if out.dtype != torch.complex64 or not out.is_contiguous() or out.numel() != int(np.prod(shape)):
            raise ValueError("out must be a contiguous complex64 tensor of %s elements" % (int(np.prod(shape)),))
        _check(ctx, fn(ctx, out.data_ptr(), 1 if out.is_cuda else 0))
        return out
    if out is not None:
        if out.dtype != np.complex64 or not out.flags.c_contiguous or out.size != int(np.prod(shape)):
            raise ValueError("out must be a C-contiguous complex64 array of %s elements" % (int(np.prod(shape)),))
        res = out
    else:
        res = np.empty(shape, dtype=np.complex64)
    _check(ctx, fn(ctx, res.ctypes.data, 0))
    return res


def get_object(ctx, shape, out=None):
    return _get(lib().ptycho_get_object, ctx, shape, out)


def get_probe(ctx, shape, out=None):
    return _get(lib().ptycho_get_probe, ctx, shape, out)


def get_exit_waves(ctx, shape, out=None):
    return _get(lib().ptycho_get_exit_waves, ctx, shape, out)


def fourier_residual(ctx, shape, out=None):
    return _get(lib().ptycho_fourier_residual, ctx, shape, out)


def fourier_error(ctx) -> float:
    v = C.c_double()
    _check(ctx, lib().ptycho_fourier_error(ctx, C.byref(v)))
    return v.value


def simulate(ctx, shape, out=None):
    if out is not None and _is_torch(out):
        _check(ctx, lib().ptycho_simulate(ctx, out.data_ptr(), 1))
        return out
    res = np.empty(shape, dtype=np.float32)
    _check(ctx, lib().ptycho_simulate(ctx, res.ctypes.data, 0))
    return res


def fourier_error_noalloc(object, probe, positions, amplitudes, stream=None) -> float:
    """ptycho_fourier_error_noalloc: E from caller-owned device buffers with no
    device allocation inside the call.  object [ny, nx] and probe [K, M, M] are
    complex64 torch CUDA tensors, amplitudes a float32 torch CUDA tensor
    [J, M, M] of sqrt(I) in FFT order (negative = masked), positions host
    [J, 2] (y, x)."""
    import torch
    assert object.is_cuda and probe.is_cuda and amplitudes.is_cuda
    o = torch.view_as_real(object.contiguous())
    p = torch.view_as_real(probe.contiguous())
    a = amplitudes.contiguous()
    pos = np.ascontiguousarray(positions, dtype=np.float32)
    K, M = int(probe.shape[0]), int(probe.shape[-1])
    v = C.c_double()
    rc = lib().ptycho_fourier_error_noalloc(o.data_ptr(), int(object.shape[0]), int(object.shape[1]), p.data_ptr(),
                                            M, K, pos.ctypes.data, int(pos.shape[0]), a.data_ptr(), C.byref(v),
                                            stream)
    _check(None, rc)
    return v.value


def iteration(ctx) -> int:
    return lib().ptycho_iteration(ctx)


def launch_count(ctx) -> int:
    return lib().ptycho_launch_count(ctx)


def cluster_size(ctx) -> int:
    return lib().ptycho_cluster_size(ctx)


def set_profiling(ctx, enabled: bool) -> None:
    _check(ctx, lib().ptycho_set_profiling(ctx, 1 if enabled else 0))


def get_profile(ctx) -> dict:
    buf = (KernelStat * 64)()
    n = C.c_int()
    _check(ctx, lib().ptycho_get_profile(ctx, buf, 64, C.byref(n)))
    return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, bytes=buf[i].bytes)
            for i in range(min(n.value, 64))}


def destroy(ctx) -> None:
    if ctx:
        lib().ptycho_destroy(ctx)


# ------------------------------------------------------------ convenience

class Reconstruction:
    """One reconstruction context: the paper's step API (init / step / resobj /
    resprobe / post) as methods.  Arrays in and out are numpy (host) unless a
    torch CUDA tensor is given."""

    def __init__(self, M, K, J, obj_shape, **params):
        stream = params.pop("stream", None)
        self.params = default_params(M=M, K=K, J=J, obj_ny=obj_shape[0], obj_nx=obj_shape[1], **params)
        if stream is not None:
            self.params.stream = stream
        self.M, self.K, self.J = M, K, J
        self.obj_shape = tuple(obj_shape)
        self.ctx = create(self.params)

    def set_data(self, intensities, positions):
        set_data(self.ctx, intensities, positions)

    def set_positions(self, positions):
        set_positions(self.ctx, positions)

    def set_data_raw(self, raw, positions, center, saturation_bits=0, threshold=0.0, rot90=0):
        """Raw detector frames [J, H, W] (uint16, uint32 or float32; numpy or
        torch, host or GPU): cropped around center (y, x), saturated pixels
        masked, values below threshold zeroed, rotated by rot90 quarter turns
        (counter-clockwise) about the zero frequency; see ptycho_set_data_raw."""
        if _is_torch(raw):
            name = str(raw.dtype).replace("torch.", "")
            if name not in RAW_DTYPES:
                raise ValueError("raw frames must be uint16, uint32 or float32")
            raw = raw.contiguous()
            ptr, dev, keep = raw.data_ptr(), int(raw.is_cuda), raw
            if not raw.is_cuda:
                keep = raw.numpy()
                ptr = keep.ctypes.data
        else:
            keep = np.ascontiguousarray(raw)
            name = str(keep.dtype)
            if name not in RAW_DTYPES:
                raise ValueError("raw frames must be uint16, uint32 or float32")
            ptr, dev = keep.ctypes.data, 0
        J, H, W = raw.shape
        pp = Preprocess(H, W, RAW_DTYPES[name], float(center[0]), float(center[1]), int(saturation_bits),
                        float(threshold), int(rot90))
        pp_ptr, _, keep_p = _ptr_in(np.asarray(positions, dtype=np.float32))
        _check(self.ctx, lib().ptycho_set_data_raw(self.ctx, ptr, C.byref(pp), pp_ptr, dev))

    def set_init(self, object=None, probe=None):
        set_init(self.ctx, object, probe)

    def iterate(self, alg, n_iter=1):
        iterate(self.ctx, alg, n_iter)

    def checkpoint(self):
        """Everything a run needs to resume bit for bit: object, probe,
        iteration index, the positions (as refined) and (DM) the exit waves
        (host arrays)."""
        state = {"object": self.get_object(), "probe": self.get_probe(), "iteration": self.iteration,
                 "positions": self.get_positions()}
        try:
            state["exit_waves"] = self.get_exit_waves()
        except PtychoError as e:
            if e.name != "STATE":
                raise
        return state

    def restore(self, state):
        """Resume from :meth:`checkpoint` (data must already be set)."""
        if "positions" in state:
            self.set_positions(state["positions"])
        self.set_init(state["object"], state["probe"])
        _check(self.ctx, lib().ptycho_set_iteration(self.ctx, int(state["iteration"])))
        if "exit_waves" in state:
            p, dev, keep = _ptr_in(state["exit_waves"])
            _check(self.ctx, lib().ptycho_set_exit_waves(self.ctx, p, dev))

    def orthogonalize_probe(self):
        """Rotate the probe modes into orthogonal modes of decreasing power now."""
        _check(self.ctx, lib().ptycho_orthogonalize_probe(self.ctx))

    def set_likelihood(self, likelihood):
        """LSQML noise model from the next iteration on: "amplitude" or "poisson"."""
        v = LIKELIHOOD[likelihood] if isinstance(likelihood, str) else int(likelihood)
        _check(self.ctx, lib().ptycho_set_likelihood(self.ctx, v))

    def set_log(self, fn=None, error_every=0):
        """Log sink fn(level, message) (level 0 error, 1 progress), called
        from inside the library calls; error_every > 0 adds a progress report
        with the Fourier error every error_every iterations.  fn=None removes it."""
        if fn is None:
            self._log_cb = None
            _check(self.ctx, lib().ptycho_set_log(self.ctx, LOG_FN(), None, int(error_every)))
            return
        self._log_cb = LOG_FN(lambda user, level, msg: fn(int(level), msg.decode()))  # kept alive with the context
        _check(self.ctx, lib().ptycho_set_log(self.ctx, self._log_cb, None, int(error_every)))

    def set_wait_limit(self, polls):
        """Polls of a cluster-transpose wait in the Fourier kernels before it
        gives up (default 1 << 20; 0 gives up at once)."""
        _check(self.ctx, lib().ptycho_set_wait_limit(self.ctx, int(polls)))

    def get_object(self, out=None):
        return get_object(self.ctx, self.obj_shape, out)

    def get_probe(self, out=None):
        return get_probe(self.ctx, (self.K, self.M, self.M), out)

    def get_exit_waves(self, out=None):
        return get_exit_waves(self.ctx, (self.J, self.K, self.M, self.M), out)

    def fourier_residual(self, out=None):
        return fourier_residual(self.ctx, (self.J, self.K, self.M, self.M), out)

    def fourier_error(self):
        return fourier_error(self.ctx)

    def refine_positions(self, step=1.0, max_shift=0.5):
        """One position-correction step (sub-pixel contexts): every position
        moves by step * clamp(s, +-max_shift) px, s the shift that best
        explains the current Fourier residual (see ptycho_refine_positions)."""
        _check(self.ctx, lib().ptycho_refine_positions(self.ctx, float(step), float(max_shift)))

    def get_positions(self):
        """Current positions [J, 2] (y, x), float32."""
        out = np.empty((self.J, 2), np.float32)
        _check(self.ctx, lib().ptycho_get_positions(self.ctx, out.ctypes.data))
        return out

    def simulate(self, out=None):
        return simulate(self.ctx, (self.J, self.M, self.M), out)

    @property
    def epie_cluster(self):
        """CTAs of the ePIE sweep (with sub-pixel positions: of its
        per-position Fourier pass)."""
        return lib().ptycho_epie_cluster_size(self.ctx)

    @property
    def iteration(self):
        return iteration(self.ctx)

    @property
    def launch_count(self):
        return launch_count(self.ctx)

    @property
    def memory_used(self):
        """Bytes of device memory the context holds."""
        return lib().ptycho_memory_used(self.ctx)

    @property
    def cluster(self):
        return cluster_size(self.ctx)

    def set_profiling(self, on=True):
        set_profiling(self.ctx, on)

    def get_profile(self):
        return get_profile(self.ctx)

    def close(self):
        if self.ctx:
            destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_fma_peak(stream=None) -> tuple[float, float, int]:
    """ptycho_fp32_fma_peak: (TFLOP/s, ms of the timed run, SM count) of the
    FP32 fused multiply-add microbenchmark on the current device."""
    tf, ms, sms = C.c_double(), C.c_double(), C.c_int()
    _check(None, lib().ptycho_fp32_fma_peak(C.byref(tf), C.byref(ms), C.byref(sms), stream))
    return tf.value, ms.value, sms.value


def autotune(M: int, K: int) -> tuple[int, float]:
    """ptycho_autotune: (fastest cluster size, ms per scan position) for (M, K)."""
    best = C.c_int()
    ms = C.c_double()
    _check(None, lib().ptycho_autotune(M, K, C.byref(best), C.byref(ms)))
    return best.value, ms.value


def autotune_engine(M: int, K: int) -> tuple[str, int, float]:
    """ptycho_autotune_engine: (faster transform engine, the register FFT's
    best cluster size, ms per scan position of the winner) for (M, K)."""
    eng, best, ms = C.c_int(), C.c_int(), C.c_double()
    _check(None, lib().ptycho_autotune_engine(M, K, C.byref(eng), C.byref(best), C.byref(ms)))
    name = {v: k for k, v in FFT_ENGINE.items()}[eng.value]
    return name, best.value, ms.value


class _Member(Reconstruction):
    """A batch member: a context owned by its batch (never destroyed here)."""

    def __init__(self, handle, M, K, J, obj_shape):
        self.ctx = C.c_void_p(handle)
        self.M, self.K, self.J = M, K, J
        self.obj_shape = tuple(obj_shape)

    def close(self):
        self.ctx = None


class Batch:
    """ptycho_batch_*: N reconstructions of unequal size, one CUDA graph per
    iteration.  ``members`` is a list of dicts with keys M, K, J, obj_shape and
    optional parameters (cluster, reg, lsqml_beta, probe_start, istore)."""

    def __init__(self, members, stream=None, group_bytes=None):
        n = len(members)
        arr = (Params * n)()
        for i, m in enumerate(members):
            kw = {k: v for k, v in m.items() if k not in ("M", "K", "J", "obj_shape")}
            arr[i] = default_params(M=m["M"], K=m["K"], J=m["J"], obj_ny=m["obj_shape"][0],
                                    obj_nx=m["obj_shape"][1], **kw)
        h = C.c_void_p()
        rc = lib().ptycho_batch_create(C.byref(h), n, arr, stream)
        if rc != 0:
            raise PtychoError(rc, (lib().ptycho_batch_last_error(None) or b"").decode())
        self.h = h
        self.members = [_Member(lib().ptycho_batch_member(h, i), m["M"], m["K"], m["J"], m["obj_shape"])
                        for i, m in enumerate(members)]
        if group_bytes is not None:
            self.set_group_bytes(group_bytes)

    def set_group_bytes(self, nbytes):
        """Working-set budget of a group of concurrently running members
        (<= 0: all members at once)."""
        self._check(lib().ptycho_batch_set_group_bytes(self.h, int(nbytes)))

    def set_lanes(self, lanes):
        """lanes > 0: members in that many chains run side by side (largest
        work first, each to the least-loaded chain); 0: groups."""
        self._check(lib().ptycho_batch_set_lanes(self.h, int(lanes)))

    @property
    def lanes(self):
        return lib().ptycho_batch_lanes(self.h)

    def autotune(self, alg="lsqml", n_iter=2):
        """Time n_iter iterations under each candidate schedule (group budgets
        and lanes) and keep the fastest: (group bytes, lanes or 0, ms per
        iteration).  The timed iterations are real iterations of every member."""
        gb, ln, ms = C.c_longlong(), C.c_int(), C.c_double()
        a = ALGS[alg] if isinstance(alg, str) else int(alg)
        self._check(lib().ptycho_batch_autotune(self.h, a, int(n_iter), C.byref(gb), C.byref(ln), C.byref(ms)))
        return gb.value, ln.value, ms.value

    def groups(self):
        """Group index of every member under the current budget."""
        n = len(self.members)
        out = (C.c_int * n)()
        ng = lib().ptycho_batch_groups(self.h, out)
        if ng < 0:
            raise PtychoError(-1, "bad batch")
        return list(out)

    def _check(self, rc):
        if rc != 0:
            raise PtychoError(rc, (lib().ptycho_batch_last_error(self.h) or b"").decode())

    def iterate(self, alg, n_iter=1):
        a = ALGS[alg] if isinstance(alg, str) else int(alg)
        self._check(lib().ptycho_batch_iterate(self.h, a, int(n_iter)))

    def synchronize(self):
        self._check(lib().ptycho_batch_synchronize(self.h))

    @property
    def kernels_per_iteration(self):
        return lib().ptycho_batch_kernels_per_iteration(self.h)

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.ctx = None
            lib().ptycho_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """ptycho_net_*: the warm-start encoder-decoder.  Frames and targets are
    float32 torch CUDA tensors ([B,128,128] detector-centred intensities,
    [B,2,64,64] amplitude/phase); parameters are host float32 arrays."""

    def __init__(self, seed=0, max_batch=64, stream=None, f32_activations=False, cuda_cores=False):
        h = C.c_void_p()
        flags = (1 if f32_activations else 0) | (2 if cuda_cores else 0)
        rc = lib().ptycho_net_create(C.byref(h), seed, max_batch, flags, stream)
        if rc != 0:
            raise PtychoError(rc, (lib().ptycho_net_last_error(None) or b"").decode())
        self.h = h
        self.max_batch = max_batch

    def _check(self, rc):
        if rc != 0:
            raise PtychoError(rc, (lib().ptycho_net_last_error(self.h) or b"").decode())

    @property
    def num_params(self):
        return lib().ptycho_net_num_params(self.h)

    def get_params(self):
        out = np.empty(self.num_params, np.float32)
        self._check(lib().ptycho_net_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        self._check(lib().ptycho_net_set_params(self.h, p.ctypes.data))

    def predict(self, frames, out):
        self._check(lib().ptycho_net_predict(self.h, frames.data_ptr(), int(frames.shape[0]), out.data_ptr()))
        return out

    def gradients(self, frames, targets):
        g = np.empty(self.num_params, np.float32)
        L = C.c_double()
        self._check(lib().ptycho_net_gradients(self.h, frames.data_ptr(), targets.data_ptr(), int(frames.shape[0]),
                                               g.ctypes.data, C.byref(L)))
        return L.value, g

    def train_step(self, frames, targets, lr, want_loss=False):
        L = C.c_double()
        self._check(lib().ptycho_net_train_step(self.h, frames.data_ptr(), targets.data_ptr(), int(frames.shape[0]),
                                                C.c_float(lr), C.byref(L) if want_loss else None))
        return L.value if want_loss else None

    def close(self):
        if getattr(self, "h", None):
            lib().ptycho_net_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def object_patches(rec, out):
    """ptycho_object_patches: central 64x64 amplitude/phase of rec's object at
    every position, into a float32 torch CUDA tensor [J,2,64,64]."""
    _check(rec.ctx, lib().ptycho_object_patches(rec.ctx, out.data_ptr()))
    return out


def warm_start(rec, net):
    """ptycho_warm_start: stitch the network's predicted patches into rec's object."""
    _check(rec.ctx, lib().ptycho_warm_start(rec.ctx, net.h))


def to_pixels(wavelength_m: float, distance_m: float, det_pixel_m: float, M: int, length_m: float) -> float:
    """Length in object-plane pixels for a far-field geometry: the object pixel
    is dx = lambda z / (M dx_d) (Sec. 3.2, Listing 1 parameters)."""
    return length_m / (wavelength_m * distance_m / (M * det_pixel_m))
