"""Thin ctypes binding of libmlx (include/mlx.h): argument marshalling only.

Every step of the transform pair, the nonlinear term and the implicit solve runs
in the CUDA library; this module converts torch CUDA tensors to device pointers
and the current torch stream to a cudaStream_t, and turns negative return codes
into MlxError.  There is no CPU fallback: if libmlx.so is missing, loading fails
with an error that says how to build it.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlx.so")

FP64, FP32, BF16X3 = 0, 1, 2
CHOP_LINEAR, CHOP_TWOTHIRDS = 0, 1
NONLIN_NONE, NONLIN_FKPP, NONLIN_VORTEX = 0, 1, 2
STEP_FEBE_HALF, STEP_FEBE_FULL, STEP_ABCN = 0, 1, 2

# Entry points declared in include/mlx.h (checked by the CPU test suite).
EXPORTS = ("mlx_strerror", "mlx_last_cuda_error", "mlx_create", "mlx_destroy", "mlx_query",
           "mlx_get_nodes", "mlx_forward", "mlx_backward", "mlx_nonlinear",
           "mlx_implicit_setup", "mlx_implicit_solve", "mlx_advance",
           "mlx_timing", "mlx_timing_read", "mlx_kernel_count", "mlx_kernel_name",
           "mlx_set_tuning", "mlx_device_status", "mlx_forward_noalloc",
           "mlx_vortex_setup", "mlx_lap_h_solve",
           "mlx_batch_create", "mlx_batch_destroy", "mlx_batch_advance", "mlx_autotune")


class MlxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nphi", ctypes.c_int), ("nz", ctypes.c_int),
                ("nr_c", ctypes.c_int), ("nphi_c", ctypes.c_int), ("nz_c", ctypes.c_int),
                ("ell", ctypes.c_double), ("lz", ctypes.c_double),
                ("precision", ctypes.c_int), ("chop_policy", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nphi", ctypes.c_int), ("nz", ctypes.c_int),
                ("nc", ctypes.c_int), ("M", ctypes.c_int), ("Kz", ctypes.c_int), ("K", ctypes.c_int),
                ("n_phys", ctypes.c_longlong), ("n_spec", ctypes.c_longlong),
                ("precision", ctypes.c_int), ("ell", ctypes.c_double), ("lz", ctypes.c_double)]


_lib = None


def load():
    """Load libmlx.so once (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmlx.so not built: run `python -m paper_2609_18026_b300.build` "
                           "(the CUDA library is required; there is no CPU path)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.mlx_strerror.restype = ctypes.c_char_p
    lib.mlx_strerror.argtypes = [i]
    lib.mlx_last_cuda_error.restype = ctypes.c_char_p
    lib.mlx_last_cuda_error.argtypes = [vp]
    lib.mlx_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    lib.mlx_destroy.argtypes = [vp]
    lib.mlx_query.argtypes = [vp, ctypes.POINTER(Info)]
    lib.mlx_get_nodes.argtypes = [vp, vp, vp, vp]
    lib.mlx_forward.argtypes = [vp, vp, vp, vp]
    lib.mlx_backward.argtypes = [vp, vp, vp, vp]
    lib.mlx_nonlinear.argtypes = [vp, i, ctypes.POINTER(d), i, vp, vp, vp]
    lib.mlx_implicit_setup.argtypes = [vp, d, d, i, d, vp]
    lib.mlx_implicit_solve.argtypes = [vp, i, vp, vp, vp, vp, vp]
    lib.mlx_advance.argtypes = [vp, i, ctypes.POINTER(d), i, vp, vp, i, i, vp]
    lib.mlx_timing.argtypes = [vp, i]
    lib.mlx_timing_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(d)]
    lib.mlx_kernel_count.argtypes = []
    lib.mlx_set_tuning.argtypes = [vp, ctypes.c_char_p, i]
    lib.mlx_device_status.argtypes = [vp]
    lib.mlx_forward_noalloc.argtypes = [vp, vp, vp, vp]
    lib.mlx_vortex_setup.argtypes = [vp, vp]
    lib.mlx_lap_h_solve.argtypes = [vp, vp, vp, vp]
    lib.mlx_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
    lib.mlx_batch_destroy.argtypes = [vp]
    lib.mlx_batch_advance.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(vp),
                                      ctypes.POINTER(vp), i, i, vp]
    lib.mlx_autotune.argtypes = [vp, i, ctypes.POINTER(d), i, ctypes.c_char_p, ctypes.POINTER(i), vp]
    lib.mlx_kernel_name.argtypes = [i]
    lib.mlx_kernel_name.restype = ctypes.c_char_p
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    lib.mlx_strerror.restype = ctypes.c_char_p
    lib.mlx_last_cuda_error.restype = ctypes.c_char_p
    lib.mlx_kernel_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """One solver context (mlx_ctx) for a grid and precision."""

    def __init__(self, nr, nphi, nz, ell, lz=6.283185307179586, precision=FP64,
                 chop_policy=CHOP_LINEAR, nr_c=0, nphi_c=0, nz_c=0, stream=None):
        self.lib = load()
        p = Params(nr, nphi, nz, nr_c, nphi_c, nz_c, float(ell), float(lz), precision, chop_policy)
        h = ctypes.c_void_p()
        self._h = None
        self._check(self.lib.mlx_create(ctypes.byref(p), _stream(stream), ctypes.byref(h)))
        self._h = h
        inf = Info()
        self._check(self.lib.mlx_query(self._h, ctypes.byref(inf)))
        self.info = inf
        self.nr, self.nphi, self.nz = inf.nr, inf.nphi, inf.nz
        self.nc, self.M, self.Kz, self.K = inf.nc, inf.M, inf.Kz, inf.K
        self.n_phys, self.n_spec = inf.n_phys, inf.n_spec
        self.precision = precision
        self.ell, self.lz = float(ell), float(lz)

    def _check(self, rc):
        if rc != 0:
            msg = self.lib.mlx_strerror(rc).decode()
            if self._h is not None:
                detail = self.lib.mlx_last_cuda_error(self._h).decode()
                if detail:
                    msg += ": " + detail
            raise MlxError(rc, "libmlx: %s (code %d)" % (msg, rc))

    def close(self):
        if self._h is not None:
            self.lib.mlx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- helpers -------------------------------------------------------
    @property
    def phys_dtype(self):
        import torch
        return torch.float64 if self.precision == FP64 else torch.float32

    def new_phys(self):
        import torch
        return torch.zeros((self.nz, self.nphi, self.nr), dtype=self.phys_dtype, device="cuda")

    def new_spec(self):
        import torch
        return torch.zeros(self.n_spec, dtype=torch.complex128, device="cuda")

    def nodes(self):
        import numpy as np
        x = np.zeros(self.nr)
        w = np.zeros(self.nr)
        r = np.zeros(self.nr)
        self._check(self.lib.mlx_get_nodes(self._h, x.ctypes.data_as(ctypes.c_void_p),
                                           w.ctypes.data_as(ctypes.c_void_p),
                                           r.ctypes.data_as(ctypes.c_void_p)))
        return x, w, r

    # ---- entry points --------------------------------------------------
    def forward(self, phys, spec, stream=None):
        self._check(self.lib.mlx_forward(self._h, _ptr(phys), _ptr(spec), _stream(stream)))
        return spec

    def backward(self, spec, phys, stream=None):
        self._check(self.lib.mlx_backward(self._h, _ptr(spec), _ptr(phys), _stream(stream)))
        return phys

    def nonlinear(self, kind, coeffs, spec_in, spec_out, stream=None):
        arr = (ctypes.c_double * max(1, len(coeffs)))(*coeffs)
        self._check(self.lib.mlx_nonlinear(self._h, kind, arr, len(coeffs), _ptr(spec_in),
                                           _ptr(spec_out), _stream(stream)))
        return spec_out

    def implicit_setup(self, nu, dt, nu_h=0.0, p=8, stream=None):
        self._check(self.lib.mlx_implicit_setup(self._h, float(nu), float(nu_h), int(p), float(dt),
                                                _stream(stream)))

    def implicit_solve(self, step, s, A, A_prev, out, stream=None):
        self._check(self.lib.mlx_implicit_solve(self._h, step, _ptr(s), _ptr(A), _ptr(A_prev),
                                                _ptr(out), _stream(stream)))
        return out

    def device_status(self):
        """Raise MlxError(MLX_ETIMEOUT) if a kernel gave up a bounded wait."""
        self._check(self.lib.mlx_device_status(self._h))

    def set_tuning(self, key, value):
        self._check(self.lib.mlx_set_tuning(self._h, key.encode(), int(value)))

    def vortex_setup(self, stream=None):
        self._check(self.lib.mlx_vortex_setup(self._h, _stream(stream)))

    def lap_h_solve(self, rhs, out, stream=None):
        self._check(self.lib.mlx_lap_h_solve(self._h, _ptr(rhs), _ptr(out), _stream(stream)))
        return out

    def timing(self, enable):
        self._check(self.lib.mlx_timing(self._h, int(bool(enable))))

    def timing_read(self):
        """{kernel name: (launches, total ms)} for kernels launched while timing was on."""
        out = {}
        for k in range(self.lib.mlx_kernel_count()):
            n = ctypes.c_longlong()
            ms = ctypes.c_double()
            self._check(self.lib.mlx_timing_read(self._h, k, ctypes.byref(n), ctypes.byref(ms)))
            if n.value:
                out[self.lib.mlx_kernel_name(k).decode()] = (n.value, ms.value)
        return out

    def autotune(self, kind, coeffs, cache_path=None, stream=None):
        """Pick launch shapes by timing; returns dict(bn, cpw, wpb, from_cache)."""
        arr = (ctypes.c_double * max(1, len(coeffs)))(*coeffs)
        ch = (ctypes.c_int * 4)()
        self._check(self.lib.mlx_autotune(self._h, kind, arr, len(coeffs),
                                          cache_path.encode() if cache_path else None, ch, _stream(stream)))
        return dict(bn=ch[0], cpw=ch[1], wpb=ch[2], from_cache=bool(ch[3]))

    def advance(self, kind, coeffs, state, prev_A, nsteps, start, stream=None):
        arr = (ctypes.c_double * max(1, len(coeffs)))(*coeffs)
        self._check(self.lib.mlx_advance(self._h, kind, arr, len(coeffs), _ptr(state), _ptr(prev_A),
                                         int(nsteps), int(bool(start)), _stream(stream)))
        return state


class Batch:
    """Independent contexts advanced together by one CUDA graph per step pair."""

    def __init__(self, contexts):
        self.lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = ctypes.c_void_p()
        rc = self.lib.mlx_batch_create(arr, len(self.contexts), ctypes.byref(h))
        if rc != 0:
            raise MlxError(rc, "libmlx: mlx_batch_create failed (code %d)" % rc)
        self._h = h

    def advance(self, kinds, coeffs, states, prevs, nsteps, start, stream=None):
        n = len(self.contexts)
        k = (ctypes.c_int * n)(*kinds)
        c = (ctypes.c_double * n)(*coeffs)
        s = (ctypes.c_void_p * n)(*[t.data_ptr() for t in states])
        p = (ctypes.c_void_p * n)(*[t.data_ptr() for t in prevs])
        rc = self.lib.mlx_batch_advance(self._h, k, c, s, p, int(nsteps), int(bool(start)), _stream(stream))
        if rc != 0:
            raise MlxError(rc, "libmlx: mlx_batch_advance failed (code %d): %s" % (
                rc, self.lib.mlx_strerror(rc).decode()))

    def close(self):
        if self._h is not None:
            self.lib.mlx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
