"""Plain FP64 CPU oracle for the WENO5 Teukolsky stage operator (arXiv 2010.04760).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its reference arm) may import this
package. It shares no code with the CUDA library under
``paper_2010_04760_gb300``; the C source ``teuk_oracle.c`` cites the paper
passage each routine follows.

Layout: state ``u[4, nth, nr]`` (Psi_R, Psi_I, pi_R, pi_I); coefficients
``coef[10, nth, nr]`` = b, Re K, Im K, Re Bt, Im Bt, Re C, Im C, Ath, Bth, c
(c: the pi rows' speed, equal to b in r*). Radial coordinate: r* (coords 0) or
the hyperboloidal rho (coords 1), its range in ``rs_min, rs_max`` either way.
Weight precision codes: 0 binary64, 1 binary32, 2 binary16, 3 bfloat16.

``ld_rhs`` / ``ld_rk3_step`` (``teuk_oracle_ld.c``) evolve the same discrete
problem with the state in C long double, to measure the binary64 state's own
round-off.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "teuk_oracle.c")
_LIB = os.path.join(_HERE, "libteuk_oracle.so")
_lib = None

WPREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "f64r": 4}


def build(force=False, src=_SRC, out=_LIB):
    """Compile the oracle with gcc (plain -O2, no FMA contraction, OpenMP).
    ``src``/``out`` default to this package's source and library; the
    mutation tests compile altered copies of the source to other paths."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-I", _HERE, "-o", out, src, "-lm"]
    subprocess.check_call(cmd)
    return out


class Grid(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nth", ctypes.c_int),
                ("rs_min", ctypes.c_double), ("rs_max", ctypes.c_double),
                ("M", ctypes.c_double), ("a", ctypes.c_double),
                ("s", ctypes.c_int), ("m", ctypes.c_int),
                ("eps", ctypes.c_double), ("wprec", ctypes.c_int),
                ("theta_mode", ctypes.c_int), ("scheme", ctypes.c_int),
                ("ko_sigma", ctypes.c_double), ("coords", ctypes.c_int),
                ("field", ctypes.c_int), ("S", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        # TEUK_ORACLE_LIB names a prebuilt oracle library to load instead (the
        # mutation tests run the pins against copies with planted mistakes)
        path = os.environ.get("TEUK_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        sig = {
            "orc_rstar_of_r": (D, [D, D, D]),
            "orc_r_of_rstar": (D, [D, D, D]),
            "orc_x_of_rstar": (D, [D, D, D]),
            "orc_coeff_point": (None, [D, D, D, D, I, I, I, P]),
            "orc_coeff_point_hyp": (None, [D, D, D, D, D, I, I, P]),
            "orc_rho_of_r": (D, [D, D]),
            "orc_coefficients": (None, [P, P]),
            "orc_round_w": (D, [I, D]),
            "orc_weno5_weights": (None, [I, I, P, D, P]),
            "orc_weno5_flux": (D, [I, I, P, D, P, P, P]),
            "orc_weno5_deriv_1d": (None, [P, I, D, I, I, D, I, P, P, P, P]),
            "orc_fd6_ko8_1d": (None, [P, I, D, D, I, P, P]),
            "orc_rhs": (None, [P, P, P, P]),
            "orc_rk3_step": (None, [P, P, D, P, L]),
            "orc_rk3_linear": (None, [D, D, D, L, P]),
            "orc_rk104_step": (None, [P, P, D, P, L]),
            "orc_rk104_linear": (None, [D, D, D, L, P]),
            "orc_advect_1d": (None, [P, I, D, D, L, I, I, D]),
            "orc_observe": (None, [P, P, D, P, P]),
            "orc_num_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def grid(nr, nth, rs_min, rs_max, M=1.0, a=0.0, s=0, m=0, eps=1e-6, wprec="fp64", theta_mode=0,
         scheme=0, ko_sigma=0.01, coords=0, field=0, S=20.0):
    """Grid description. coords 1 (hyperboloidal) always evolves Phi."""
    w = WPREC[wprec] if isinstance(wprec, str) else int(wprec)
    if int(coords) == 1:
        field = 1
    return Grid(nr, nth, rs_min, rs_max, M, a, s, m, eps, w, int(theta_mode), int(scheme),
                float(ko_sigma), int(coords), int(field), float(S))


def rho_of_r(r, S):
    return _load().orc_rho_of_r(float(r), float(S))


def horizon_rho(M, a, S):
    """rho of the outer horizon r_+ = M + sqrt(M^2 - a^2)."""
    return rho_of_r(M + np.sqrt(max(M * M - a * a, 0.0)), S)


def num_threads():
    return _load().orc_num_threads()


def rstar_of_r(r, M=1.0, a=0.0):
    return _load().orc_rstar_of_r(r, M, a)


def r_of_rstar(rs, M=1.0, a=0.0):
    return _load().orc_r_of_rstar(rs, M, a)


def x_of_rstar(rs, M=1.0, a=0.0):
    """r - r_+ at r* (resolved where it is far below the spacing of r)."""
    return _load().orc_x_of_rstar(rs, M, a)


def coeff_point(r, th, M, a, s, m, field=0):
    out = np.zeros(10)
    _load().orc_coeff_point(r, th, M, a, s, m, int(field), _ptr(out))
    return out


def coeff_point_hyp(rho, th, M, a, S, s, m):
    out = np.zeros(10)
    _load().orc_coeff_point_hyp(rho, th, M, a, S, s, m, _ptr(out))
    return out


def coefficients(g):
    coef = np.zeros((10, g.nth, g.nr))
    _load().orc_coefficients(ctypes.byref(g), _ptr(coef))
    return coef


def round_w(wprec, x):
    w = WPREC[wprec] if isinstance(wprec, str) else int(wprec)
    return _load().orc_round_w(w, float(x))


def weno5_weights(f5, dir, wprec="fp64", eps=1e-6):
    w = WPREC[wprec] if isinstance(wprec, str) else int(wprec)
    f5 = _f64(f5)
    out = np.zeros(3)
    _load().orc_weno5_weights(w, dir, _ptr(f5), eps, _ptr(out))
    return out


def fd6_ko8_1d(f, h, sigma=0.01, periodic=True, bc=None):
    """bc: 0 edge copy, 1 periodic, 2 polynomial extrapolation (default from
    ``periodic``)."""
    f = _f64(f)
    D, Q = np.zeros(f.size), np.zeros(f.size)
    bc = int(periodic) if bc is None else int(bc)
    _load().orc_fd6_ko8_1d(_ptr(f), f.size, h, sigma, bc, _ptr(D), _ptr(Q))
    return D, Q


def weno5_deriv_1d(f, h, dir, wprec="fp64", eps=1e-6, periodic=True, force_w=None,
                   return_wq=False, bc=None):
    """bc: 0 edge copy, 1 periodic, 2 polynomial extrapolation (default from
    ``periodic``)."""
    w = WPREC[wprec] if isinstance(wprec, str) else int(wprec)
    f = _f64(f)
    n = f.size
    D = np.zeros(n)
    fw = None if force_w is None else _f64(force_w)
    wo = np.zeros((n, 3)) if return_wq else None
    qo = np.zeros((n, 3)) if return_wq else None
    bc = int(periodic) if bc is None else int(bc)
    _load().orc_weno5_deriv_1d(_ptr(f), n, h, dir, w, eps, bc,
                               None if fw is None else _ptr(fw), _ptr(D),
                               None if wo is None else _ptr(wo),
                               None if qo is None else _ptr(qo))
    if return_wq:
        return D, wo, qo
    return D


def rhs(g, coef, u):
    coef, u = _f64(coef), _f64(u)
    F = np.zeros_like(u)
    _load().orc_rhs(ctypes.byref(g), _ptr(coef), _ptr(u), _ptr(F))
    return F


def rk3_step(g, coef, dt, u, nsteps=1):
    coef = _f64(coef)
    u = _f64(u).copy()
    _load().orc_rk3_step(ctypes.byref(g), _ptr(coef), dt, _ptr(u), int(nsteps))
    return u


def rk104_step(g, coef, dt, u, nsteps=1):
    coef = _f64(coef)
    u = _f64(u).copy()
    _load().orc_rk104_step(ctypes.byref(g), _ptr(coef), dt, _ptr(u), int(nsteps))
    return u


def rk104_linear(lam, dt, nsteps, y0=1.0 + 0.0j):
    y = np.array([np.real(y0), np.imag(y0)], dtype=np.float64)
    _load().orc_rk104_linear(float(np.real(lam)), float(np.imag(lam)), dt, int(nsteps), _ptr(y))
    return complex(y[0], y[1])


def rk3_linear(lam, dt, nsteps, y0=1.0 + 0.0j):
    y = np.array([np.real(y0), np.imag(y0)], dtype=np.float64)
    _load().orc_rk3_linear(float(np.real(lam)), float(np.imag(lam)), dt, int(nsteps), _ptr(y))
    return complex(y[0], y[1])


def advect_1d(f, h, dt, nsteps, dir=1, wprec="fp64", eps=1e-6):
    w = WPREC[wprec] if isinstance(wprec, str) else int(wprec)
    f = _f64(f).copy()
    _load().orc_advect_1d(_ptr(f), f.size, h, dt, int(nsteps), dir, w, eps)
    return f


def observe(g, u, rs_ext):
    u = _f64(u)
    wave = np.zeros((g.nth, 2))
    hor = np.zeros((g.nth, 6))
    _load().orc_observe(ctypes.byref(g), _ptr(u), rs_ext, _ptr(wave), _ptr(hor))
    return wave, hor


# ---------------------------------------------------------------------------
# Extended-precision state (teuk_oracle_ld.c): the same right-hand side and
# SSP-RK(3,3) step with the state, weights and fluxes in C long double
# (binary128 on aarch64, the x87 64-bit-significand format on x86-64), for
# measuring the binary64 state's own round-off. Arrays are numpy longdouble,
# which is C long double on both.
# ---------------------------------------------------------------------------
_SRC_LD = os.path.join(_HERE, "teuk_oracle_ld.c")
_LIB_LD = os.path.join(_HERE, "libteuk_oracle_ld.so")
_lib_ld = None


def build_ld(force=False, src=_SRC_LD, out=_LIB_LD):
    """Compile the extended-precision oracle (same flags as the binary64 one;
    ``src``/``out`` as for ``build``)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-I", _HERE, "-o", out, src, "-lm"])
    return out


def _load_ld():
    global _lib_ld
    if _lib_ld is None:
        # TEUK_ORACLE_LD_LIB: a prebuilt copy to load instead (mutation tests)
        lib = ctypes.CDLL(os.environ.get("TEUK_ORACLE_LD_LIB") or build_ld())
        I, D, L, P = ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_void_p
        sig = {"orc_ld_mant_dig": (I, []),
               "orc_ld_weno5_flux": (None, [I, P, P, P]),
               "orc_ld_rhs": (I, [P, P, P, P]),
               "orc_ld_rk3_step": (I, [P, P, D, P, L])}
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib_ld = lib
    return _lib_ld


def _ld(a):
    return np.ascontiguousarray(a, dtype=np.longdouble)


def ld_mant_dig():
    """Significand bits of the extended state (113 binary128, 64 x87)."""
    return _load_ld().orc_ld_mant_dig()


def ld_weno5_flux(f5, dir, eps=1e-6):
    """WENO5 flux of five long double values (dir +1: f_{j-2..j+2}, dir -1:
    f_{j-1..j+3}; the interface j+1/2 either way)."""
    f5 = _ld(f5)
    e = np.array([eps], dtype=np.longdouble)
    out = np.zeros(1, dtype=np.longdouble)
    _load_ld().orc_ld_weno5_flux(int(dir), _ptr(f5), _ptr(e), _ptr(out))
    return out[0]


def _ld_supported(g):
    if g.scheme != 0 or g.theta_mode != 0:
        raise ValueError("the extended-precision oracle covers WENO5 with centred theta only")


def ld_rhs(g, coef, u):
    _ld_supported(g)
    coef, u = _f64(coef), _ld(u)
    F = np.zeros(u.shape, dtype=np.longdouble)
    _load_ld().orc_ld_rhs(ctypes.byref(g), _ptr(coef), _ptr(u), _ptr(F))
    return F


def ld_rk3_step(g, coef, dt, u, nsteps=1):
    _ld_supported(g)
    coef = _f64(coef)
    u = _ld(u).copy()
    _load_ld().orc_ld_rk3_step(ctypes.byref(g), _ptr(coef), float(dt), _ptr(u), int(nsteps))
    return u
