"""GB300 (sm_103a) mixed-precision WENO5 Teukolsky solver (arXiv 2010.04760).

Thin Python binding of the C ABI declared in ``include/teuk.h``: every
function here has the C function's name and only marshals arguments; all
arithmetic runs in the CUDA library ``libteuk.so`` built next to this file by
``paper_2010_04760_gb300.build``. There is no CPU fallback: if the library is
missing, every call raises.

Device arrays are passed as CUDA ``torch`` tensors (float64, contiguous) or as
raw integer device pointers; host arrays as numpy float64 arrays. Streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers, or None.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libteuk.so")

(TEUK_OK, TEUK_ERR_ARG, TEUK_ERR_CUDA, TEUK_ERR_NONFINITE, TEUK_ERR_TIMEOUT, TEUK_ERR_STATE,
 TEUK_ERR_HOST) = range(7)
TEUK_W_FP64, TEUK_W_FP32, TEUK_W_FP16, TEUK_W_BF16 = range(4)
TEUK_THETA_CENTERED4, TEUK_THETA_WENO5 = 0, 1
TEUK_RK_SSP33, TEUK_RK_SSP104 = 0, 1
TEUK_SCHEME_WENO5, TEUK_SCHEME_FD6_KO8 = 0, 1
TEUK_COORDS_RSTAR, TEUK_COORDS_HYPERBOLOIDAL = 0, 1
TEUK_FIELD_PSI, TEUK_FIELD_PHI = 0, 1
TEUK_LAUNCH_AUTO, TEUK_LAUNCH_STAGES, TEUK_LAUNCH_FUSED = 0, 1, 2
WPREC = {"fp64": TEUK_W_FP64, "fp32": TEUK_W_FP32, "fp16": TEUK_W_FP16, "bf16": TEUK_W_BF16}


class TeukError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class teuk_params(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("rstar_min", ctypes.c_double), ("rstar_max", ctypes.c_double),
                ("M", ctypes.c_double), ("a", ctypes.c_double),
                ("s", ctypes.c_int), ("m", ctypes.c_int),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("eps", ctypes.c_double), ("wprec", ctypes.c_int),
                ("theta_mode", ctypes.c_int), ("rk", ctypes.c_int),
                ("scheme", ctypes.c_int), ("ko_sigma", ctypes.c_double),
                ("coords", ctypes.c_int), ("field", ctypes.c_int),
                ("hyp_S", ctypes.c_double)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2010_04760_gb300.build.build() "
                               "(needs nvcc); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I, I64, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        PP = ctypes.POINTER(teuk_params)
        sig = {
            "teuk_status_str": (ctypes.c_char_p, [I]),
            "teuk_last_error": (ctypes.c_char_p, []),
            "teuk_check_params": (I, [PP]),
            "teuk_horizon_rho": (I, [D, D, D, P]),
            "teuk_stable_dt": (I, [PP, P]),
            "teuk_coeff_count": (S, [PP]),
            "teuk_build_coefficients": (I, [PP, D, P]),
            "teuk_stage_dev": (I, [PP, D, P, P, P, P, I, P]),
            "teuk_step_dev": (I, [PP, D, P, P, P, I64, P]),
            "teuk_step_dev_static": (I, [PP, D, P, P, I64, P]),
            "teuk_fp64_fma_rate": (I, [P, P]),
            "teuk_create": (I, [PP, P, P]),
            "teuk_destroy": (I, [P]),
            "teuk_get_info": (I, [P, PP, P, P]),
            "teuk_set_initial": (I, [P, P, P]),
            "teuk_set_state": (I, [P, P, D]),
            "teuk_set_gaussian": (I, [P, D, D, P, I, ctypes.c_uint64]),
            "teuk_get_state": (I, [P, P, P]),
            "teuk_set_state_async": (I, [P, P, D]),
            "teuk_get_state_async": (I, [P, P]),
            "teuk_synchronize": (I, [P]),
            "teuk_step": (I, [P, I64]),
            "teuk_observe": (I, [P, D, P, P, P]),
            "teuk_check_finite": (I, [P]),
            "teuk_state_dev": (I, [P, P]),
            "teuk_set_launch": (I, [P, I, D]),
            "teuk_get_launch": (I, [P, P, P, P]),
            "teuk_test_withhold": (I, [P]),
            "teuk_batch_create": (I, [PP, I, P, I, P]),
            "teuk_batch_destroy": (I, [P]),
            "teuk_batch_set_state": (I, [P, I, P, D]),
            "teuk_batch_get_state": (I, [P, I, P, P]),
            "teuk_batch_step": (I, [P, I64]),
            "teuk_batch_get_info": (I, [P, I, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    """Names of the functions include/teuk.h declares (parsed from the header)."""
    import re
    hdr = os.path.join(_HERE, "..", "include", "teuk.h")
    with open(hdr) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|teuk_status|size_t)\s+(teuk_\w+)\s*\(",
                                 text, flags=re.M)))


def _check(st):
    if st != TEUK_OK:
        msg = lib().teuk_last_error().decode() or lib().teuk_status_str(st).decode()
        raise TeukError(st, msg)


def _dptr(x, need=0, what="device array"):
    """Device pointer of a CUDA float64 tensor holding at least `need` values
    (checked), or of a raw integer pointer (the caller vouches for its size)."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        if not x.is_cuda or x.dtype.__str__() != "torch.float64" or not x.is_contiguous():
            raise ValueError("device arrays must be contiguous CUDA float64 tensors")
        if x.numel() < need:
            raise ValueError(f"{what}: needs {need} float64 values, the tensor has {x.numel()}")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError("expected a CUDA tensor or an integer device pointer")


def _nodes(p):
    return int(p.nr) * int(p.ntheta)


def _host_in(a, n, what):
    """A C-contiguous float64 view or copy of host array a, which must hold
    exactly n values (the library reads n)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"{what}: expected {n} float64 values, got {a.size}")
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _host_out(out, n, what):
    """Check a caller's output array: writable C-contiguous float64 of n values."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.flags.writeable and out.size == n):
        raise ValueError(f"{what}: out must be a writable C-contiguous float64 array of "
                         f"{n} values")
    return out.ctypes.data_as(ctypes.c_void_p)


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)


def make_params(nr, ntheta, rstar_min=None, rstar_max=None, M=1.0, a=0.0, s=0, m=0,
                cfl=0.5, dt=0.0, eps=1e-6, wprec="fp64", theta_mode=TEUK_THETA_CENTERED4,
                rk=TEUK_RK_SSP33, scheme=TEUK_SCHEME_WENO5, ko_sigma=0.01,
                coords=TEUK_COORDS_RSTAR, field=None, hyp_S=20.0):
    """teuk_params with defaults: r* in [-100, 300] M; on the hyperboloidal
    slices the whole range [rho_+, S] (rho_+ from the library) and the field
    Phi."""
    w = WPREC[wprec] if isinstance(wprec, str) else int(wprec)
    hyp = coords == TEUK_COORDS_HYPERBOLOIDAL
    if rstar_min is None:
        rstar_min = teuk_horizon_rho(M, a, hyp_S) if hyp else -100.0
    if rstar_max is None:
        rstar_max = hyp_S if hyp else 300.0
    if field is None:
        field = TEUK_FIELD_PHI if hyp else TEUK_FIELD_PSI
    return teuk_params(nr, ntheta, rstar_min, rstar_max, M, a, s, m, cfl, dt, eps, w, theta_mode,
                       rk, scheme, ko_sigma, coords, field, hyp_S)


def params_from_workload(wl, **over):
    kw = dict(nr=wl.nr, ntheta=wl.nth, rstar_min=wl.rs_min, rstar_max=wl.rs_max, M=wl.M, a=wl.a,
              s=wl.s, m=wl.m, cfl=wl.cfl, eps=wl.eps, wprec=wl.wprec,
              coords=getattr(wl, "coords", TEUK_COORDS_RSTAR),
              field=getattr(wl, "field", None), hyp_S=getattr(wl, "S", 20.0))
    kw.update(over)
    return make_params(**kw)


# ---- C-ABI functions (same names) ------------------------------------------

def teuk_status_str(st):
    return lib().teuk_status_str(st).decode()


def teuk_last_error():
    return lib().teuk_last_error().decode()


def teuk_check_params(p):
    return lib().teuk_check_params(ctypes.byref(p))


def teuk_horizon_rho(M, a, S):
    """rho of the outer horizon on the hyperboloidal slices."""
    out = ctypes.c_double()
    _check(lib().teuk_horizon_rho(float(M), float(a), float(S), ctypes.byref(out)))
    return out.value


horizon_rho = teuk_horizon_rho


def teuk_stable_dt(p):
    out = ctypes.c_double()
    _check(lib().teuk_stable_dt(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def teuk_coeff_count(p):
    return lib().teuk_coeff_count(ctypes.byref(p))


def teuk_build_coefficients(p, dt):
    n = teuk_coeff_count(p)
    if n == 0:
        _check(lib().teuk_check_params(ctypes.byref(p)))
    out = np.zeros((n // (p.ntheta * p.nr), p.ntheta, p.nr))
    _check(lib().teuk_build_coefficients(ctypes.byref(p), dt, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def teuk_stage_dev(p, dt, coef_dev, u_n, u_prev, u_out, stage, stream=None):
    n, nc = 4 * _nodes(p), teuk_coeff_count(p)
    _check(lib().teuk_stage_dev(ctypes.byref(p), dt, _dptr(coef_dev, nc, "coef_dev"),
                                _dptr(u_n, n, "u_n"), _dptr(u_prev, n, "u_prev"),
                                _dptr(u_out, n, "u_out"), int(stage), _stream(stream)))


def teuk_step_dev(p, dt, coef_dev, u_dev, work_dev, nsteps, stream=None):
    n, nc = 4 * _nodes(p), teuk_coeff_count(p)
    scratch = 3 if p.rk == TEUK_RK_SSP104 else 2
    _check(lib().teuk_step_dev(ctypes.byref(p), dt, _dptr(coef_dev, nc, "coef_dev"),
                               _dptr(u_dev, n, "u_dev"), _dptr(work_dev, scratch * n, "work_dev"),
                               int(nsteps), _stream(stream)))


def teuk_fp64_fma_rate(stream=None):
    """Measured binary64 lane-FMAs per second of the current device."""
    out = ctypes.c_double()
    _check(lib().teuk_fp64_fma_rate(_stream(stream), ctypes.byref(out)))
    return out.value


TEUK_STATIC_MAX_NODES = 131072


def teuk_step_dev_static(p, dt, coef_dev, u_dev, nsteps, stream=None):
    """teuk_step_dev without caller scratch: the stage buffers are a fixed
    array inside the library (grids up to TEUK_STATIC_MAX_NODES nodes)."""
    _check(lib().teuk_step_dev_static(ctypes.byref(p), dt,
                                      _dptr(coef_dev, teuk_coeff_count(p), "coef_dev"),
                                      _dptr(u_dev, 4 * _nodes(p), "u_dev"), int(nsteps),
                                      _stream(stream)))


class Handle:
    """Owner of a teuk_handle*; the methods are the handle calls of teuk.h."""

    def __init__(self, ptr, p):
        self.ptr = ptr
        self.p = p

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.ptr:
            lib().teuk_destroy(self.ptr)
            self.ptr = None


def teuk_create(p, stream=None):
    h = ctypes.c_void_p()
    _check(lib().teuk_create(ctypes.byref(p), _stream(stream), ctypes.byref(h)))
    return Handle(h, p)


def teuk_destroy(h):
    h.close()


def teuk_get_info(h):
    p, dt, t = teuk_params(), ctypes.c_double(), ctypes.c_double()
    _check(lib().teuk_get_info(h.ptr, ctypes.byref(p), ctypes.byref(dt), ctypes.byref(t)))
    return p, dt.value, t.value


def teuk_set_initial(h, psi, pi):
    """psi, pi: complex arrays [ntheta, nr]."""
    ps = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
    pc = np.ascontiguousarray(np.asarray(pi, dtype=np.complex128))
    if ps.size != _nodes(h.p) or pc.size != _nodes(h.p):
        raise ValueError(f"psi and pi need {_nodes(h.p)} complex values each")
    _check(lib().teuk_set_initial(h.ptr, ps.ctypes.data_as(ctypes.c_void_p),
                                  pc.ctypes.data_as(ctypes.c_void_p)))


def teuk_set_gaussian(h, rc, width, coeffs=None, nl=None, seed=0):
    """coeffs: complex amplitudes per l (from max(|s|, |m|) upward), or None to
    draw them from SplitMix64(seed) (then nl terms)."""
    if coeffs is not None:
        c = np.asarray(coeffs, dtype=np.complex128)
        arr = np.ascontiguousarray(np.stack([c.real, c.imag], axis=-1).ravel())
        n = c.size
        ptr = arr.ctypes.data_as(ctypes.c_void_p)
    else:
        n, ptr = int(nl or 1), None
    _check(lib().teuk_set_gaussian(h.ptr, float(rc), float(width), ptr, n, int(seed)))


def teuk_set_state(h, u, t=0.0):
    arr, ptr = _host_in(u, 4 * _nodes(h.p), "teuk_set_state")
    _check(lib().teuk_set_state(h.ptr, ptr, float(t)))


def teuk_get_state(h, out=None):
    if out is None:
        out = np.empty((4, h.p.ntheta, h.p.nr))
    ptr = _host_out(out, 4 * _nodes(h.p), "teuk_get_state")
    t = ctypes.c_double()
    _check(lib().teuk_get_state(h.ptr, ptr, ctypes.byref(t)))
    return out, t.value


def teuk_set_state_async(h, u, t=0.0):
    """Enqueue the host-to-device copy of u (keep u alive and unchanged, and
    preferably page-locked, until the stream has passed the copy)."""
    arr = np.ascontiguousarray(u, dtype=np.float64)
    if arr is not u:
        raise ValueError("teuk_set_state_async needs a C-contiguous float64 array "
                         "(a temporary copy would be freed before the copy runs)")
    if arr.size != 4 * _nodes(h.p):
        raise ValueError(f"teuk_set_state_async: expected {4 * _nodes(h.p)} values")
    _check(lib().teuk_set_state_async(h.ptr, arr.ctypes.data_as(ctypes.c_void_p), float(t)))


def teuk_get_state_async(h, out):
    """Enqueue the device-to-host copy of the state into out (defined after
    teuk_synchronize)."""
    ptr = _host_out(out, 4 * _nodes(h.p), "teuk_get_state_async")
    _check(lib().teuk_get_state_async(h.ptr, ptr))


def teuk_synchronize(h):
    _check(lib().teuk_synchronize(h.ptr))


def teuk_step(h, nsteps):
    _check(lib().teuk_step(h.ptr, int(nsteps)))


def teuk_observe(h, rstar_ext):
    wave = np.empty((h.p.ntheta, 2))
    hor = np.empty((h.p.ntheta, 6))
    t = ctypes.c_double()
    _check(lib().teuk_observe(h.ptr, float(rstar_ext), wave.ctypes.data_as(ctypes.c_void_p),
                              hor.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t)))
    return wave, hor, t.value


def teuk_check_finite(h):
    return lib().teuk_check_finite(h.ptr)


def teuk_set_launch(h, mode, wait_seconds=2.0):
    _check(lib().teuk_set_launch(h.ptr, int(mode), float(wait_seconds)))


def teuk_get_launch(h):
    """(mode, wait_seconds, 1 if teuk_step uses the fused step else 0)."""
    mode, wait, k = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    _check(lib().teuk_get_launch(h.ptr, ctypes.byref(mode), ctypes.byref(wait),
                                 ctypes.byref(k)))
    return mode.value, wait.value, k.value


def teuk_test_withhold(h):
    _check(lib().teuk_test_withhold(h.ptr))


def teuk_state_dev(h):
    ptr = ctypes.c_void_p()
    _check(lib().teuk_state_dev(h.ptr, ctypes.byref(ptr)))
    return ptr.value


class Batch:
    """Owner of a teuk_batch*; members keep the order of the parameter list."""

    def __init__(self, ptr, ps):
        self.ptr = ptr
        self.ps = list(ps)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.ptr:
            lib().teuk_batch_destroy(self.ptr)
            self.ptr = None


def teuk_batch_create(ps, stream=None, autotune=True):
    arr = (teuk_params * len(ps))(*ps)
    b = ctypes.c_void_p()
    _check(lib().teuk_batch_create(arr, len(ps), _stream(stream), int(bool(autotune)),
                                   ctypes.byref(b)))
    return Batch(b, ps)


def teuk_batch_destroy(b):
    b.close()


def _member(b, k):
    if not 0 <= int(k) < len(b.ps):
        raise IndexError(f"member {k} of a batch of {len(b.ps)}")
    return b.ps[int(k)]


def teuk_batch_set_state(b, k, u, t=0.0):
    arr, ptr = _host_in(u, 4 * _nodes(_member(b, k)), "teuk_batch_set_state")
    _check(lib().teuk_batch_set_state(b.ptr, int(k), ptr, float(t)))


def teuk_batch_get_state(b, k, out=None):
    p = _member(b, k)
    if out is None:
        out = np.empty((4, p.ntheta, p.nr))
    ptr = _host_out(out, 4 * _nodes(p), "teuk_batch_get_state")
    t = ctypes.c_double()
    _check(lib().teuk_batch_get_state(b.ptr, int(k), ptr, ctypes.byref(t)))
    return out, t.value


def teuk_batch_step(b, nsteps):
    _check(lib().teuk_batch_step(b.ptr, int(nsteps)))


def teuk_batch_get_info(b, k):
    dt, t = ctypes.c_double(), ctypes.c_double()
    seg, ctas = ctypes.c_int(), ctypes.c_int()
    _check(lib().teuk_batch_get_info(b.ptr, int(k), ctypes.byref(dt), ctypes.byref(t),
                                     ctypes.byref(seg), ctypes.byref(ctas)))
    return dt.value, t.value, seg.value, ctas.value
