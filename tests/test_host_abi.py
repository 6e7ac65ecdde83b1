"""Host-side tests of the C ABI (no GPU): the library loads and exports every
symbol include/teuk.h declares, arguments are validated, and the host
coefficient generator (independent code) agrees with the oracle."""
import ctypes
import os

import numpy as np
import pytest

import oracle as o
import paper_2010_04760_gb300 as T
from paper_2010_04760_gb300 import build as B
from paper_2010_04760_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_library_exports_every_declared_symbol():
    names = T.declared_symbols()
    assert len(names) >= 18
    L = T.lib()
    for n in names:
        assert hasattr(L, n), n


def test_status_strings():
    names = [T.teuk_status_str(st) for st in range(7)]
    assert all(names) and len(set(names)) == 7
    assert T.teuk_status_str(7) == "unknown status"


def test_check_params_limits_are_inclusive():
    assert T.teuk_check_params(T.make_params(7, 262140)) == T.TEUK_OK
    assert T.teuk_check_params(T.make_params(7, 5)) == T.TEUK_OK


@pytest.mark.parametrize("field,value", [("nr", 6), ("ntheta", 4), ("a", 1.5), ("M", 0.0),
                                         ("s", 3), ("eps", 0.0), ("wprec", 7), ("cfl", 0.0),
                                         ("rstar_max", -200.0), ("dt", -1.0), ("theta_mode", 9),
                                         ("m", 65), ("ntheta", 262141)])
def test_check_params_rejects(field, value):
    p = T.make_params(64, 16)
    setattr(p, field, value)
    assert T.teuk_check_params(p) == T.TEUK_ERR_ARG
    assert T.teuk_last_error()


def test_check_params_accepts_workloads():
    for wl in [I.SCHW_SCALAR, I.KERR_GRAV, I.EXTREMAL_SCALAR, I.TAIL_SCALAR]:
        assert T.teuk_check_params(T.params_from_workload(wl)) == T.TEUK_OK


def test_stable_dt_rule():
    p = T.make_params(256, 32, a=0.0, s=0, m=0, cfl=0.5)
    dt = T.teuk_stable_dt(p)
    h = 400.0 / 255
    assert 0.0 < dt < 0.5 * h        # the upwind part alone allows cfl * h / b
    p.dt = 0.01
    assert T.teuk_stable_dt(p) == 0.01


@pytest.mark.parametrize("a,s,m", [(0.0, 0, 0), (0.999, -2, 2), (1.0, 0, 0), (0.4, -1, 1),
                                   (0.7, -2, 3)])
def test_coefficients_agree_with_oracle(a, s, m):
    nr, nth, rs0, rs1, dt = 40, 12, -60.0, 120.0, 0.07
    p = T.make_params(nr, nth, rs0, rs1, 1.0, a, s, m)
    got = T.teuk_build_coefficients(p, dt)
    co = o.coefficients(o.grid(nr, nth, rs0, rs1, 1.0, a, s, m))
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth = co[:9]
    h = (rs1 - rs0) / (nr - 1)
    dth = np.pi / nth
    tol = dict(rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(got[0], dt * b / (6 * h), **tol)
    np.testing.assert_allclose(got[1], dt * Kr / (6 * h), **tol)
    np.testing.assert_allclose(got[2], dt * Ki / (6 * h), **tol)
    np.testing.assert_allclose(got[3], dt * Br, **tol)
    np.testing.assert_allclose(got[4], dt * Bi, **tol)
    np.testing.assert_allclose(got[5], dt * Ci, **tol)
    # theta planes applied to a pole-parity-respecting field reproduce
    # Ath Psi_thth + Bth Psi_th + Re C Psi from the oracle's ghost-cell operator
    rng = np.random.default_rng(0)
    psi = rng.standard_normal((nth, nr))
    sig = 1.0 if (m + s) % 2 == 0 else -1.0
    acc = np.zeros((nth, nr))
    for k in range(-2, 3):
        rows = np.clip(np.arange(nth) + k, 0, nth - 1)
        acc += got[8 + k] * psi[rows]
    ext = np.concatenate([sig * psi[1::-1], psi, sig * psi[:-3:-1]])   # rows -2..nth+1
    nb = [ext[2 + k:2 + k + nth] for k in range(-2, 3)]
    th1 = (nb[0] - 8 * nb[1] + 8 * nb[3] - nb[4]) / (12 * dth)
    th2 = (-nb[0] + 16 * nb[1] - 30 * nb[2] + 16 * nb[3] - nb[4]) / (12 * dth ** 2)
    exp_ = dt * (Ath * th2 + Bth * th1 + Cr * psi)
    np.testing.assert_allclose(acc, exp_, rtol=1e-8, atol=1e-10 * np.max(np.abs(exp_)))


def test_theta_weno_option_adds_a_plane():
    p = T.make_params(64, 16, a=0.5, s=-2, m=1, theta_mode=1)
    assert T.teuk_check_params(p) == T.TEUK_OK
    assert T.teuk_coeff_count(p) == 12 * 64 * 16
    c1 = T.teuk_build_coefficients(p, 0.1)
    p0 = T.make_params(64, 16, a=0.5, s=-2, m=1, theta_mode=0)
    c0 = T.teuk_build_coefficients(p0, 0.1)
    np.testing.assert_array_equal(c1[:6], c0[:6])
    co = o.coefficients(o.grid(64, 16, -100.0, 300.0, 1.0, 0.5, -2, 1))
    np.testing.assert_allclose(c1[11], 0.1 * co[8] / (6 * np.pi / 16), rtol=1e-9, atol=1e-15)


def test_ssprk104_step_rule_and_stage_step():
    p3 = T.make_params(128, 16, a=0.5, s=-2, m=2)
    p10 = T.make_params(128, 16, a=0.5, s=-2, m=2, rk=1)
    assert abs(T.teuk_stable_dt(p10) / T.teuk_stable_dt(p3) - 2.8) < 1e-12
    # coefficients carry the forward-Euler stage step dt/6
    np.testing.assert_allclose(T.teuk_build_coefficients(p10, 0.6),
                               T.teuk_build_coefficients(p3, 0.1), rtol=1e-15, atol=0)
    bad = T.make_params(128, 16, rk=2)
    assert T.teuk_check_params(bad) == T.TEUK_ERR_ARG


def test_fd6_scheme_argument_rules():
    assert T.teuk_check_params(T.make_params(64, 16, scheme=1)) == T.TEUK_OK
    assert T.teuk_check_params(T.make_params(64, 16, scheme=2)) == T.TEUK_ERR_ARG
    assert T.teuk_check_params(T.make_params(64, 16, scheme=1, theta_mode=1)) == T.TEUK_ERR_ARG
    assert T.teuk_check_params(T.make_params(64, 16, scheme=1, ko_sigma=-0.1)) == T.TEUK_ERR_ARG


def test_build_coefficients_rejects_bad_dt():
    p = T.make_params(64, 16)
    with pytest.raises(T.TeukError):
        T.teuk_build_coefficients(p, 0.0)


def _check_planes_against_oracle(p, co, dt, coords):
    """The kernel planes of p against the oracle's coefficients co: radial
    planes scaled by dt/(6h), the rest by dt (plane 12 = the pi rows' speed
    on the hyperboloidal slices)."""
    got = T.teuk_build_coefficients(p, dt)
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth, c = co
    h = (p.rstar_max - p.rstar_min) / (p.nr - 1)
    scale = np.max(np.abs(co), axis=(1, 2))
    for k, (plane, ref) in enumerate([(0, dt * b / (6 * h)), (1, dt * Kr / (6 * h)),
                                      (2, dt * Ki / (6 * h)), (3, dt * Br), (4, dt * Bi),
                                      (5, dt * Ci)]):
        np.testing.assert_allclose(got[plane], ref, rtol=1e-9, atol=1e-13 * dt * max(scale) / h)
    if coords == 1:
        np.testing.assert_allclose(got[12], dt * c / (6 * h), rtol=1e-9, atol=1e-14)
        assert np.all(got[11] == 0.0)
    _check_theta_planes(got, co, p.s, p.m, dt)


def _check_theta_planes(got, co, s, m, dt):
    """The five theta planes applied to a field with the pole parity give
    dt (Ath Psi_thth + Bth Psi_th + Re C Psi) of the oracle's ghost-row
    operator (fourth-order centred differences)."""
    nth, nr = got.shape[1:]
    Cr, Ath, Bth = co[5], co[7], co[8]
    dth = np.pi / nth
    psi = np.random.default_rng(0).standard_normal((nth, nr))
    sig = 1.0 if (m + s) % 2 == 0 else -1.0
    acc = np.zeros((nth, nr))
    for k in range(-2, 3):
        rows = np.clip(np.arange(nth) + k, 0, nth - 1)
        acc += got[8 + k] * psi[rows]
    ext = np.concatenate([sig * psi[1::-1], psi, sig * psi[:-3:-1]])   # rows -2..nth+1
    nb = [ext[2 + k:2 + k + nth] for k in range(-2, 3)]
    th1 = (nb[0] - 8 * nb[1] + 8 * nb[3] - nb[4]) / (12 * dth)
    th2 = (-nb[0] + 16 * nb[1] - 30 * nb[2] + 16 * nb[3] - nb[4]) / (12 * dth ** 2)
    exp_ = dt * (Ath * th2 + Bth * th1 + Cr * psi)
    np.testing.assert_allclose(acc, exp_, rtol=1e-8, atol=1e-10 * np.max(np.abs(exp_)))


@pytest.mark.parametrize("a,s,m", [(0.0, 0, 0), (1.0, -2, 0), (0.7, -2, 2), (0.3, 1, -1),
                                   (0.95, 2, 3)])
def test_hyperboloidal_coefficients_agree_with_oracle(a, s, m):
    """Sec. 2.2 slices: the host's closed forms (analytic d b/d rho) against
    the oracle's (complex-step d b/d rho), horizon to scri."""
    nr, nth, S, dt = 48, 10, 20.0, 0.01
    p = T.make_params(nr, nth, a=a, s=s, m=m, coords=T.TEUK_COORDS_HYPERBOLOIDAL, hyp_S=S)
    assert T.teuk_check_params(p) == T.TEUK_OK, T.teuk_last_error()
    assert T.teuk_coeff_count(p) == 13 * nr * nth
    g = o.grid(nr, nth, p.rstar_min, p.rstar_max, 1.0, a, s, m, coords=1, S=S)
    _check_planes_against_oracle(p, o.coefficients(g), dt, 1)


@pytest.mark.parametrize("a,s,m", [(0.0, 0, 0), (0.999, -2, 2), (0.4, -1, 1), (0.7, 2, 3)])
def test_rescaled_field_coefficients_agree_with_oracle(a, s, m):
    nr, nth, rs0, rs1, dt = 40, 12, -60.0, 120.0, 0.07
    p = T.make_params(nr, nth, rs0, rs1, 1.0, a, s, m, field=T.TEUK_FIELD_PHI)
    g = o.grid(nr, nth, rs0, rs1, 1.0, a, s, m, field=1)
    _check_planes_against_oracle(p, o.coefficients(g), dt, 0)


def test_hyperboloidal_argument_rules():
    H = T.TEUK_COORDS_HYPERBOLOIDAL
    ok = T.make_params(64, 16, a=0.6, s=-2, m=1, coords=H)
    assert T.teuk_check_params(ok) == T.TEUK_OK
    rhop = T.horizon_rho(1.0, 0.6, 20.0)
    assert abs(ok.rstar_min - rhop) < 1e-15 and ok.rstar_max == 20.0
    assert T.teuk_check_params(T.make_params(64, 16, a=0.6, coords=H, scheme=1)) == T.TEUK_OK
    assert T.teuk_check_params(T.make_params(64, 16, a=0.6, coords=H, theta_mode=1)) == T.TEUK_OK
    bad = [dict(field=T.TEUK_FIELD_PSI), dict(scheme=1, theta_mode=1),
           dict(hyp_S=0.5, rstar_min=0.0, rstar_max=0.0), dict(rstar_min=rhop * 0.999),
           dict(rstar_max=20.001),
           dict(coords=2), dict(field=3)]
    for kw in bad:
        p = T.make_params(64, 16, a=0.6, s=-2, m=1, **{**dict(coords=H), **kw})
        assert T.teuk_check_params(p) == T.TEUK_ERR_ARG, kw
        assert T.teuk_last_error()
    # a sub-range strictly inside [rho_+, S] is fine
    assert T.teuk_check_params(T.make_params(64, 16, 2.0, 15.0, a=0.6, coords=H)) == T.TEUK_OK


def test_hyperboloidal_time_step_uses_the_larger_speed():
    """dt = cfl / max(max(|b|, |c|)/h + sqrt(kappa)) (the pi rows' speed c is
    the larger one near the horizon, where b vanishes)."""
    H = T.TEUK_COORDS_HYPERBOLOIDAL
    p = T.make_params(256, 16, a=1.0, s=-2, m=0, coords=H, cfl=0.5)
    dt = T.teuk_stable_dt(p)
    g = o.grid(256, 16, p.rstar_min, p.rstar_max, 1.0, 1.0, -2, 0, coords=1, S=20.0)
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth, c = o.coefficients(g)
    h = (p.rstar_max - p.rstar_min) / 255
    dth = np.pi / 16
    kap = Ath * (16 / 3) / dth ** 2 + np.abs(Bth) * 1.5 / dth + np.hypot(Cr, Ci)
    lam = np.max(np.maximum(np.abs(b), np.abs(c)) / h + np.sqrt(kap))
    assert abs(dt - 0.5 / lam) < 1e-9 * dt


def test_batches_reject_mixed_coordinates():
    """Argument checks run before any device call, so this needs no GPU."""
    ps = [T.make_params(64, 16), T.make_params(64, 16, coords=T.TEUK_COORDS_HYPERBOLOIDAL)]
    with pytest.raises(T.TeukError):
        T.teuk_batch_create(ps, stream=0, autotune=False)
    assert "coords" in T.teuk_last_error()


def test_params_struct_layout_matches_the_header(tmp_path):
    """The binding's teuk_params has the header's field order, offsets and
    size (a C program compiled against include/teuk.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [f[0] for f in T.teuk_params._fields_]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("{n} %zu\\n", offsetof(teuk_params, {n}));\n' for n in names)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "teuk.h"\nint main(void) {\n'
                   + body + '    printf("sizeof %zu\\n", sizeof(teuk_params));\n    return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for n in names:
        assert int(got[n]) == getattr(T.teuk_params, n).offset, n
    assert int(got["sizeof"]) == ctypes.sizeof(T.teuk_params)


def _c_client(tmp_path):
    """Builds tests/c/teuk_c_client.c against include/teuk.h and libteuk.so."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(T.LIB_PATH)
    exe = str(tmp_path / "teuk_c_client")
    subprocess.check_call([cc, "-O2", "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "c", "teuk_c_client.c"), "-o", exe,
                           "-L", libdir, "-lteuk", "-lm", "-Wl,-rpath," + libdir])
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join(
        [p for p in ("/usr/local/cuda/lib64", env.get("LD_LIBRARY_PATH", "")) if p])

    def run(*args):
        out = subprocess.run([exe, *args], capture_output=True, text=True, env=env)
        assert out.returncode == 0, out.stderr
        return dict(line.split(None, 1) for line in out.stdout.splitlines())
    return run


def test_plain_c_client_of_the_abi(tmp_path):
    """A C program using only include/teuk.h gets the same time step and
    coefficient array as the Python binding, and a status (with a message)
    for an invalid parameter set."""
    got = _c_client(tmp_path)()
    p = T.params_from_workload(I.KERR_GRAV, wprec="fp32")
    dt = T.teuk_stable_dt(p)
    assert float(got["dt"]) == dt
    assert int(got["coef_count"]) == T.teuk_coeff_count(p)
    assert float(got["coef_abs_sum"]) == pytest.approx(np.abs(T.teuk_build_coefficients(p, dt)).sum(),
                                                       rel=1e-12)   # summation order
    assert int(got["bad_status"]) == T.TEUK_ERR_ARG and got["bad_message_nonempty"] == "1"
    # the whole hyperboloidal slice from the range [0, 0], rho_+ filled in by
    # the library (the client never computes it)
    rhop = I.horizon_rho(1.0, 1.0, 20.0)
    assert float(got["horizon_rho"]) == pytest.approx(rhop, rel=1e-15)
    q = T.make_params(512, 16, rhop, 20.0, 1.0, 1.0, -2, 0, wprec="fp32",
                      coords=T.TEUK_COORDS_HYPERBOLOIDAL)
    assert float(got["hyp_dt"]) == T.teuk_stable_dt(q)


def test_hyperboloidal_default_range():
    """rstar_min == rstar_max == 0 on the hyperboloidal slices is the whole
    slice [rho_+, S] for every call that takes parameters; in r* it is an
    empty range and an error."""
    rhop = T.teuk_horizon_rho(1.0, 0.6, 20.0)
    assert rhop == pytest.approx(I.horizon_rho(1.0, 0.6, 20.0), rel=1e-15)
    full = T.make_params(64, 8, rhop, 20.0, 1.0, 0.6, -2, 1, coords=T.TEUK_COORDS_HYPERBOLOIDAL)
    zero = T.make_params(64, 8, 0.0, 0.0, 1.0, 0.6, -2, 1, coords=T.TEUK_COORDS_HYPERBOLOIDAL)
    assert T.teuk_check_params(zero) == T.TEUK_OK
    assert T.teuk_stable_dt(zero) == T.teuk_stable_dt(full)
    np.testing.assert_array_equal(T.teuk_build_coefficients(zero, 0.01),
                                  T.teuk_build_coefficients(full, 0.01))
    assert T.teuk_check_params(T.make_params(64, 8, 0.0, 0.0)) == T.TEUK_ERR_ARG
    for bad in [(0.0, 1.0, 20.0), (1.0, 1.5, 20.0), (1.0, 0.5, 0.5)]:
        with pytest.raises(T.TeukError):
            T.teuk_horizon_rho(*bad)


_HOST_OOM_CHILD = r"""
import ctypes, resource, sys
sys.path.insert(0, sys.argv[1])
import paper_2010_04760_gb300 as T
L = T.lib()
limit = 2 << 30                                   # 2 GiB of address space from here on
soft, hard = resource.getrlimit(resource.RLIMIT_AS)
used = int(open("/proc/self/statm").read().split()[0]) * resource.getpagesize()
resource.setrlimit(resource.RLIMIT_AS, (used + limit, hard))
# 4e8 nodes with a given dt: the coefficient array alone would take 35 GB
p = T.make_params(20000, 20000, dt=0.01)
h = ctypes.c_void_p(12345)
st = L.teuk_create(ctypes.byref(p), None, ctypes.byref(h))
print(st, h.value, L.teuk_last_error().decode())
"""


def test_host_allocation_failure_is_a_status():
    """A host allocation that fails inside a call comes back as
    TEUK_ERR_HOST with a message and a NULL handle; no C++ exception crosses
    the ABI (which would abort the process). The child process caps its
    address space so that the coefficient array of a 4e8-node grid cannot be
    allocated; nothing touches a GPU before that point."""
    import subprocess
    import sys
    T.lib()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _HOST_OOM_CHILD, root], capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    st, handle, msg = out.stdout.strip().split(None, 2)
    assert int(st) == T.TEUK_ERR_HOST
    assert handle == "None"
    assert msg == "teuk_create: host memory exhausted"


class _FakeCudaTensor:
    """Stands in for a CUDA float64 tensor in the binding's argument checks."""

    def __init__(self, n, dtype="torch.float64", cuda=True, contiguous=True):
        self.n, self.dtype, self.is_cuda, self._c = n, dtype, cuda, contiguous

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x1000


def test_binding_checks_array_sizes_before_calling_the_library():
    """The binding refuses arrays that are too small (or of the wrong kind)
    before any pointer reaches the library, so a size mistake in Python is
    an exception, never an access outside a buffer."""
    assert T._dptr(_FakeCudaTensor(10), 10).value == 0x1000
    with pytest.raises(ValueError, match="needs 11"):
        T._dptr(_FakeCudaTensor(10), 11, "u_out")
    for bad in (_FakeCudaTensor(10, dtype="torch.float32"), _FakeCudaTensor(10, cuda=False),
                _FakeCudaTensor(10, contiguous=False)):
        with pytest.raises(ValueError):
            T._dptr(bad, 1)
    assert T._dptr(12345, 10**9).value == 12345          # raw pointers: the caller's word
    a, _ = T._host_in(np.zeros((4, 3, 7)), 84, "u")
    assert a.size == 84
    with pytest.raises(ValueError, match="expected 84"):
        T._host_in(np.zeros((4, 3, 6)), 84, "u")
    T._host_out(np.zeros((4, 3, 7)), 84, "out")
    for bad in (np.zeros(83), np.zeros(84, dtype=np.float32), np.zeros((84, 2))[:, 0]):
        with pytest.raises(ValueError):
            T._host_out(bad, 84, "out")
    ro = np.zeros(84)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        T._host_out(ro, 84, "out")


def test_missing_library_fails_loudly_with_no_cpu_fallback(tmp_path):
    """Without the CUDA library every binding call raises; nothing computes on
    the CPU in its place."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = (
        "import sys; sys.path.insert(0, sys.argv[1])\n"
        "import paper_2010_04760_gb300 as T\n"
        "T.LIB_PATH = sys.argv[2]\n"
        "try:\n"
        "    T.teuk_check_params(T.make_params(16, 8))\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    print('no error')\n")
    out = subprocess.run([sys.executable, "-c", child, root, str(tmp_path / "absent.so")],
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised:") and "no CPU fallback" in out.stdout


def test_product_code_never_touches_the_oracle():
    """The library, its binding and the input module neither import, load nor
    name the oracle package (the oracle is test infrastructure)."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2010_04760_gb300")
    pat = re.compile(r"(import\s+oracle|from\s+oracle|teuk_oracle|orc_|libteuk_oracle)")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not pat.search(text), os.path.join(dirpath, f)


def test_fd6_radial_planes_carry_sixty_h():
    """The FD6 + KO8 kernel forms 60 h D (the sixth-order stencil's own
    normalisation, Sec. 3.1.1), so its radial planes (b, Re K, Im K) carry
    dt/(60h) where the WENO5 planes carry dt/(6h); the others are the same."""
    for coords in (T.TEUK_COORDS_RSTAR, T.TEUK_COORDS_HYPERBOLOIDAL):
        kw = dict(a=0.7, s=-2, m=1, coords=coords)
        weno = T.teuk_build_coefficients(T.make_params(64, 8, **kw), 0.01)
        fd6 = T.teuk_build_coefficients(T.make_params(64, 8, scheme=1, **kw), 0.01)
        radial = [0, 1, 2] + ([12] if coords == T.TEUK_COORDS_HYPERBOLOIDAL else [])
        for k in range(weno.shape[0]):
            if k in radial:
                np.testing.assert_allclose(fd6[k], weno[k] / 10.0, rtol=1e-15, atol=0)
            else:
                np.testing.assert_array_equal(fd6[k], weno[k])
