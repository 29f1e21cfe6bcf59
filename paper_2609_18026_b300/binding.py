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
CHOP_LINEAR, CHOP_TWOTHIRDS, CHOP_NYQUIST = 0, 1, 2
LOGPROXY_PRESCRIBE, LOGPROXY_SOLVE = 0, 1
NONLIN_NONE, NONLIN_FKPP, NONLIN_VORTEX = 0, 1, 2
STEP_FEBE_HALF, STEP_FEBE_FULL, STEP_ABCN = 0, 1, 2

# Entry points declared in include/mlx.h (checked by the CPU test suite).
EXPORTS = ("mlx_strerror", "mlx_last_cuda_error", "mlx_create", "mlx_destroy", "mlx_query",
           "mlx_get_nodes", "mlx_forward", "mlx_backward", "mlx_nonlinear",
           "mlx_implicit_setup", "mlx_implicit_solve", "mlx_advance",
           "mlx_timing", "mlx_timing_read", "mlx_kernel_count", "mlx_kernel_name",
           "mlx_set_tuning", "mlx_device_status", "mlx_forward_noalloc",
           "mlx_diag", "mlx_state_bytes", "mlx_get_state", "mlx_set_state",
           "mlx_filter_setup", "mlx_filter_apply", "mlx_filter_state", "mlx_axial_energy",
           "mlx_vortex_setup", "mlx_lap_h_solve", "mlx_lap_h_solve_log", "mlx_vortex_logproxy",
           "mlx_vortex_diag",
           "mlx_batch_create", "mlx_batch_destroy", "mlx_batch_advance", "mlx_batch_set_persistent",
           "mlx_autotune",
           "mlx_sur_create", "mlx_sur_destroy", "mlx_sur_param_count", "mlx_sur_get_params",
           "mlx_sur_set_params", "mlx_sur_get_grads", "mlx_sur_get_scales", "mlx_sur_set_scales",
           "mlx_sur_propagate", "mlx_sur_observe", "mlx_sur_finalize_scales", "mlx_sur_make_pair",
           "mlx_sur_infer", "mlx_sur_train_step", "mlx_sur_advance", "mlx_sur_status")


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


class FilterParams(ctypes.Structure):
    _fields_ = [("zeta_c", ctypes.c_double), ("tau", ctypes.c_double),
                ("eps_max", ctypes.c_double), ("relax", ctypes.c_double)]


class DiagOut(ctypes.Structure):
    _fields_ = [("integral", ctypes.c_double), ("moment2", ctypes.c_double),
                ("l2w", ctypes.c_double), ("spec_l2", ctypes.c_double)]


class VortexDiagOut(ctypes.Structure):
    _fields_ = [("enstrophy", ctypes.c_double), ("peak_vorticity", ctypes.c_double)]


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
    lib.mlx_diag.argtypes = [vp, vp, ctypes.POINTER(DiagOut), vp]
    lib.mlx_filter_setup.argtypes = [vp, i, ctypes.POINTER(FilterParams)]
    lib.mlx_filter_apply.argtypes = [vp, vp, i, vp]
    lib.mlx_filter_state.argtypes = [vp, vp, vp]
    lib.mlx_axial_energy.argtypes = [vp, vp, vp, vp]
    lib.mlx_state_bytes.argtypes = [vp, i]
    lib.mlx_state_bytes.restype = ctypes.c_longlong
    lib.mlx_get_state.argtypes = [vp, i, vp, vp, ctypes.c_longlong, vp, ctypes.c_longlong, vp]
    lib.mlx_set_state.argtypes = [vp, i, vp, ctypes.c_longlong, vp, vp, ctypes.POINTER(ctypes.c_longlong), vp]
    lib.mlx_vortex_setup.argtypes = [vp, vp]
    lib.mlx_lap_h_solve.argtypes = [vp, vp, vp, vp]
    lib.mlx_lap_h_solve_log.argtypes = [vp, vp, vp, i, ctypes.POINTER(d), vp]
    lib.mlx_vortex_logproxy.argtypes = [vp, d, d, d, vp]
    lib.mlx_vortex_diag.argtypes = [vp, vp, ctypes.POINTER(VortexDiagOut), vp]
    lib.mlx_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
    lib.mlx_batch_destroy.argtypes = [vp]
    lib.mlx_batch_set_persistent.argtypes = [vp, i]
    lib.mlx_batch_advance.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(vp),
                                      ctypes.POINTER(vp), i, i, vp]
    lib.mlx_autotune.argtypes = [vp, i, ctypes.POINTER(d), i, ctypes.c_char_p, ctypes.POINTER(i), vp]
    lib.mlx_kernel_name.argtypes = [i]
    lib.mlx_kernel_name.restype = ctypes.c_char_p
    f = ctypes.c_float
    lib.mlx_sur_create.argtypes = [i, i, i, ctypes.c_ulonglong, ctypes.POINTER(vp)]
    lib.mlx_sur_destroy.argtypes = [vp]
    lib.mlx_sur_status.argtypes = [vp]
    lib.mlx_sur_param_count.argtypes = [vp]
    lib.mlx_sur_param_count.restype = ctypes.c_longlong
    for name in ("mlx_sur_get_params", "mlx_sur_set_params", "mlx_sur_get_grads"):
        getattr(lib, name).argtypes = [vp, vp]
    lib.mlx_sur_get_scales.argtypes = [vp, vp, vp]
    lib.mlx_sur_set_scales.argtypes = [vp, vp, vp]
    lib.mlx_sur_propagate.argtypes = [vp, vp, vp, vp, i, vp]
    lib.mlx_sur_observe.argtypes = [vp, vp, vp, vp, i, vp]
    lib.mlx_sur_finalize_scales.argtypes = [vp, d, d, vp]
    lib.mlx_sur_make_pair.argtypes = [vp, vp, vp, vp, i, vp, vp, vp]
    lib.mlx_sur_infer.argtypes = [vp, vp, vp, i, vp, vp]
    lib.mlx_sur_train_step.argtypes = [vp, vp, vp, vp, i, f, vp, vp]
    lib.mlx_sur_advance.argtypes = [vp, vp, vp, i, d, i, d, ctypes.POINTER(i), ctypes.POINTER(d), vp]
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

    def lap_h_solve_log(self, rhs, out, variant, c=0.0, stream=None):
        """mlx_lap_h_solve_log: returns (out, c); c is the input amplitude for
        LOGPROXY_PRESCRIBE and the solved one for LOGPROXY_SOLVE."""
        cv = ctypes.c_double(float(c))
        self._check(self.lib.mlx_lap_h_solve_log(self._h, _ptr(rhs), _ptr(out), int(variant), ctypes.byref(cv),
                                                 _stream(stream)))
        return out, cv.value

    def vortex_logproxy(self, c_psi, c_chi, Uz=0.0, stream=None):
        """Log-proxy amplitudes of (psi, chi) and the axial background (mlx_vortex_logproxy)."""
        self._check(self.lib.mlx_vortex_logproxy(self._h, float(c_psi), float(c_chi), float(Uz), _stream(stream)))

    def vortex_diag(self, state, stream=None):
        """dict(enstrophy, peak_vorticity) of a two-field vortex state (mlx_vortex_diag)."""
        o = VortexDiagOut()
        self._check(self.lib.mlx_vortex_diag(self._h, _ptr(state), ctypes.byref(o), _stream(stream)))
        return dict(enstrophy=o.enstrophy, peak_vorticity=o.peak_vorticity)

    def diag(self, spec, stream=None):
        """dict(integral, moment2, l2w, spec_l2) of a spectral scalar field (mlx_diag)."""
        o = DiagOut()
        self._check(self.lib.mlx_diag(self._h, _ptr(spec), ctypes.byref(o), _stream(stream)))
        return dict(integral=o.integral, moment2=o.moment2, l2w=o.l2w, spec_l2=o.spec_l2)

    def filter_setup(self, enable=True, zeta_c=None, tau=None, eps_max=None, relax=None):
        """Adaptive modal filter between steps (mlx_filter_setup); None = the default."""
        p = None
        if any(v is not None for v in (zeta_c, tau, eps_max, relax)):
            p = FilterParams(2.0 / 3.0 if zeta_c is None else zeta_c, 2e-2 if tau is None else tau,
                             36.0 if eps_max is None else eps_max, 0.25 if relax is None else relax)
        self._check(self.lib.mlx_filter_setup(self._h, int(bool(enable)), ctypes.byref(p) if p else None))

    def filter_apply(self, state, nfields=1, stream=None):
        self._check(self.lib.mlx_filter_apply(self._h, _ptr(state), int(nfields), _stream(stream)))
        return state

    def filter_state(self):
        """(eps[2], tail[2]) of the filter."""
        e = (ctypes.c_double * 2)()
        t = (ctypes.c_double * 2)()
        self._check(self.lib.mlx_filter_state(self._h, e, t))
        return list(e), list(t)

    def axial_energy(self, state, stream=None):
        """Kinetic energy per axial wavenumber |k| < Kz of a two-field vortex state."""
        E = (ctypes.c_double * self.Kz)()
        self._check(self.lib.mlx_axial_energy(self._h, _ptr(state), E, _stream(stream)))
        return list(E)

    def state_bytes(self, kind):
        return int(self.lib.mlx_state_bytes(self._h, kind))

    def get_state(self, kind, state, prev_A, step=0, stream=None):
        """Checkpoint image (bytes) of (state, prev_A) with a step counter."""
        n = self.state_bytes(kind)
        buf = ctypes.create_string_buffer(n)
        self._check(self.lib.mlx_get_state(self._h, kind, _ptr(state), _ptr(prev_A), int(step), buf, n,
                                           _stream(stream)))
        return buf.raw

    def set_state(self, kind, image, state, prev_A, stream=None):
        """Restore a checkpoint image into (state, prev_A); returns its step counter."""
        buf = ctypes.create_string_buffer(bytes(image), len(image))
        step = ctypes.c_longlong()
        self._check(self.lib.mlx_set_state(self._h, kind, buf, len(image), _ptr(state), _ptr(prev_A),
                                           ctypes.byref(step), _stream(stream)))
        return step.value

    def timing(self, enable):
        """0 off; 1 (or True) direct launches bracketed by events; 2 graph replays with
        event-record nodes around every kernel node."""
        self._check(self.lib.mlx_timing(self._h, int(enable)))

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

    def set_persistent(self, on):
        rc = self.lib.mlx_batch_set_persistent(self._h, int(bool(on)))
        if rc != 0:
            raise MlxError(rc, "libmlx: mlx_batch_set_persistent failed (code %d)" % rc)

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


class Surrogate:
    """Learned spectral surrogate of the vortex solver (mlx_sur): a 4-layer
    perceptron that adds the nonlinear remainder to the linear propagator."""

    def __init__(self, D, width=64, bmax=256, seed=0):
        self.lib = load()
        h = ctypes.c_void_p()
        self._h = None
        rc = self.lib.mlx_sur_create(int(D), int(width), int(bmax), int(seed), ctypes.byref(h))
        if rc != 0:
            raise MlxError(rc, "libmlx: mlx_sur_create failed: %s (code %d)" % (
                self.lib.mlx_strerror(rc).decode(), rc))
        self._h = h
        self.D, self.width, self.bmax = int(D), int(width), int(bmax)
        self.nparam = int(self.lib.mlx_sur_param_count(self._h))

    def _check(self, rc, ctx=None):
        if rc != 0:
            msg = self.lib.mlx_strerror(rc).decode()
            if ctx is not None and ctx._h is not None:
                detail = self.lib.mlx_last_cuda_error(ctx._h).decode()
                if detail:
                    msg += ": " + detail
            raise MlxError(rc, "libmlx: %s (code %d)" % (msg, rc))

    def close(self):
        if self._h is not None:
            self.lib.mlx_sur_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self):
        """Raise MlxError(MLX_ETIMEOUT) if a tensor-core kernel gave up a bounded wait."""
        self._check(self.lib.mlx_sur_status(self._h))

    def offsets(self):
        """Offsets of W1, b1, W2, b2, W3, b3, W4, b4 in the flat parameter array."""
        D, w = self.D, self.width
        sizes = [w * D, w, w * w, w, w * w, w, D * w, D]
        out, o = [], 0
        for n in sizes:
            out.append(o)
            o += n
        return out

    def get_params(self):
        import numpy as np
        a = np.zeros(self.nparam, dtype=np.float32)
        self._check(self.lib.mlx_sur_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p)))
        return a

    def set_params(self, a):
        import numpy as np
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == self.nparam
        self._check(self.lib.mlx_sur_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p)))

    def get_grads(self):
        import numpy as np
        a = np.zeros(self.nparam, dtype=np.float32)
        self._check(self.lib.mlx_sur_get_grads(self._h, a.ctypes.data_as(ctypes.c_void_p)))
        return a

    def get_scales(self):
        import numpy as np
        a = np.zeros(self.D, dtype=np.float32)
        b = np.zeros(self.D, dtype=np.float32)
        self._check(self.lib.mlx_sur_get_scales(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                b.ctypes.data_as(ctypes.c_void_p)))
        return a, b

    def set_scales(self, a, b):
        import numpy as np
        a = np.ascontiguousarray(a, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        self._check(self.lib.mlx_sur_set_scales(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                b.ctypes.data_as(ctypes.c_void_p)))

    def propagate(self, ctx, state, out, nsub, stream=None):
        self._check(self.lib.mlx_sur_propagate(ctx._h, self._h, _ptr(state), _ptr(out), int(nsub),
                                               _stream(stream)), ctx)
        return out

    def observe(self, ctx, s0, s1, nsub, stream=None):
        self._check(self.lib.mlx_sur_observe(ctx._h, self._h, _ptr(s0), _ptr(s1), int(nsub),
                                             _stream(stream)), ctx)

    def finalize_scales(self, in_floor=1e-3, out_floor=1e-3, stream=None):
        self._check(self.lib.mlx_sur_finalize_scales(self._h, float(in_floor), float(out_floor), _stream(stream)))

    def make_pair(self, ctx, s0, s1, nsub, x, t, stream=None):
        self._check(self.lib.mlx_sur_make_pair(ctx._h, self._h, _ptr(s0), _ptr(s1), int(nsub), _ptr(x),
                                               _ptr(t), _stream(stream)), ctx)

    def infer(self, X, idx, y, stream=None):
        self._check(self.lib.mlx_sur_infer(self._h, _ptr(X), _ptr(idx), int(idx.numel()), _ptr(y),
                                           _stream(stream)))
        return y

    def train_step(self, X, T, idx, lr, loss=None, stream=None):
        self._check(self.lib.mlx_sur_train_step(self._h, _ptr(X), _ptr(T), _ptr(idx), int(idx.numel()),
                                                float(lr), _ptr(loss), _stream(stream)))

    def advance(self, ctx, state, nsub, U0, judge, tol, stream=None):
        """One call; returns (accepted, residual)."""
        a = ctypes.c_int()
        r = ctypes.c_double()
        self._check(self.lib.mlx_sur_advance(ctx._h, self._h, _ptr(state), int(nsub), float(U0),
                                             int(bool(judge)), float(tol), ctypes.byref(a), ctypes.byref(r),
                                             _stream(stream)), ctx)
        return bool(a.value), r.value
