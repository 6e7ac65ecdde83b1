"""GPU parity on the hyperboloidal slices of Sec. 2.2 and for the rescaled
field Phi = r Delta^s Psi (Sec. 4): the CUDA path against the CPU oracle,
element by element, through the C ABI. The hyperboloidal grid runs from the
horizon to scri, so every case exercises the extrapolated ghosts at both ends
and the pi rows' own speed c. Tolerance as for r*: binary64 round-off of the
differently arranged stencil arithmetic, taken node by node,
|gpu - oracle| <= 1e-12 x the size of the terms entering that node
(``_local_scale``; near either end it includes the extrapolated ghosts)."""
import numpy as np
import pytest

import oracle as o
import paper_2010_04760_gb300 as T
from paper_2010_04760_gb300 import inputs as I
from _local_scale import assert_local, run_scale, stage_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
S = 20.0
H = T.TEUK_COORDS_HYPERBOLOIDAL


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    T.lib()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_dt(g, co):
    """0.5 / max(max(|b|, |c|)/h + sqrt(theta frequencies)), from the oracle."""
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth, c = co
    h = (g.rs_max - g.rs_min) / (g.nr - 1)
    dth = np.pi / g.nth
    kap = Ath * (16 / 3) / dth ** 2 + np.abs(Bth) * 1.5 / dth + np.hypot(Cr, Ci)
    return 0.5 / np.max(np.maximum(np.abs(b), np.abs(c)) / h + np.sqrt(kap))


def compare(got, exp_, scale, tol=TOL, what=""):
    assert_local(got, exp_, scale, tol, what)


def hyp_grid(nr, nth, a, s, m, wprec="fp64", lo=None, hi=None, theta_mode=0):
    lo = I.horizon_rho(1.0, a, S) if lo is None else lo
    hi = S if hi is None else hi
    g = o.grid(nr, nth, lo, hi, 1.0, a, s, m, 1e-6, wprec, theta_mode, coords=1, S=S)
    p = T.make_params(nr, nth, lo, hi, 1.0, a, s, m, wprec=wprec, theta_mode=theta_mode,
                      coords=H, hyp_S=S)
    return g, p


SHAPES = [(7, 5), (64, 8), (100, 13), (257, 33), (1000, 17)]
PHYS = [(1.0, -2, 0), (0.0, 0, 0), (0.7, -2, 2), (0.5, 1, -1)]


@pytest.mark.parametrize("theta_mode", [0, 1])
@pytest.mark.parametrize("wprec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("phys", PHYS)
def test_hyperboloidal_operator_parity(wprec, shape, phys, theta_mode):
    nr, nth = shape
    a, s, m = phys
    for smooth in (True, False):
        # rows scaled over 1e-40..1e6 and a 1e-200 region next to the horizon
        u = I.multiscale_state(nr, nth, nr * 5 + nth, smooth)
        g, p = hyp_grid(nr, nth, a, s, m, wprec, theta_mode=theta_mode)
        co = o.coefficients(g)
        F = o.rhs(g, co, u)
        coef = dev(T.teuk_build_coefficients(p, 1.0))
        ud = dev(u)
        out = torch.empty_like(ud)
        T.teuk_stage_dev(p, 1.0, coef, None, ud, out, 0)
        compare(host(out), F, stage_scale(g, co, 1.0, u, with_prev=False),
                what=f"hyp {wprec} {shape} {phys} smooth={smooth}")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("phys", PHYS)
def test_hyperboloidal_fd6_ko8_operator_parity(shape, phys):
    """The comparison scheme (Sec. 3.1.1) on the slices, where the paper makes
    its WENO-versus-dissipation comparison: FD6 derivative, KO8 term and the
    pi rows' own speed, with four extrapolated ghosts per end."""
    nr, nth = shape
    a, s, m = phys
    lo = I.horizon_rho(1.0, a, S)
    for smooth in (True, False):
        u = I.multiscale_state(nr, nth, nr * 11 + nth, smooth)
        g = o.grid(nr, nth, lo, S, 1.0, a, s, m, scheme=1, ko_sigma=0.2, coords=1, S=S)
        co = o.coefficients(g)
        p = T.make_params(nr, nth, lo, S, 1.0, a, s, m, scheme=1, ko_sigma=0.2, coords=H,
                          hyp_S=S)
        coef = dev(T.teuk_build_coefficients(p, 1.0))
        ud = dev(u)
        out = torch.empty_like(ud)
        T.teuk_stage_dev(p, 1.0, coef, None, ud, out, 0)
        compare(host(out), o.rhs(g, co, u), stage_scale(g, co, 1.0, u, with_prev=False),
                what=f"hyp fd6 {shape} {phys} smooth={smooth}")


@pytest.mark.parametrize("wprec", ["fp64", "fp32"])
def test_hyperboloidal_sub_range_parity(wprec):
    """A range strictly inside (rho_+, S): the extrapolated ghosts act at
    interior radii."""
    nr, nth = 333, 12
    u = I.random_state(nr, nth, 9)
    g, p = hyp_grid(nr, nth, 0.6, -2, 1, wprec, lo=3.0, hi=15.0)
    co = o.coefficients(g)
    coef = dev(T.teuk_build_coefficients(p, 1.0))
    ud = dev(u)
    out = torch.empty_like(ud)
    T.teuk_stage_dev(p, 1.0, coef, None, ud, out, 0)
    compare(host(out), o.rhs(g, co, u), stage_scale(g, co, 1.0, u, with_prev=False),
            what="sub-range")


@pytest.mark.parametrize("wprec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("phys", [(0.999, -2, 2), (0.0, 0, 0), (0.5, -1, 3)])
def test_rescaled_field_operator_parity_in_rstar(wprec, phys):
    a, s, m = phys
    nr, nth, rs0, rs1 = 300, 20, -60.0, 150.0
    u = I.random_state(nr, nth, 77, smooth=False)
    g = o.grid(nr, nth, rs0, rs1, 1.0, a, s, m, 1e-6, wprec, field=1)
    co = o.coefficients(g)
    p = T.make_params(nr, nth, rs0, rs1, 1.0, a, s, m, wprec=wprec, field=T.TEUK_FIELD_PHI)
    coef = dev(T.teuk_build_coefficients(p, 1.0))
    ud = dev(u)
    out = torch.empty_like(ud)
    T.teuk_stage_dev(p, 1.0, coef, None, ud, out, 0)
    compare(host(out), o.rhs(g, co, u), stage_scale(g, co, 1.0, u, with_prev=False),
            what=f"phi r* {wprec} {phys}")


def run_both(wl, wprec, nsteps, rk=0):
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, wl.M, wl.a, wl.s, wl.m, wl.eps, wprec,
               coords=1, S=wl.S)
    co = o.coefficients(g)
    dt = oracle_dt(g, co) * (2.8 if rk == 1 else 1.0)
    u0 = I.initial_data(wl)
    p = T.params_from_workload(wl, wprec=wprec, rk=rk)
    coef = dev(T.teuk_build_coefficients(p, dt))
    ud = dev(u0)
    work = torch.empty(3, 4, wl.nth, wl.nr, dtype=torch.float64, device="cuda")
    T.teuk_step_dev(p, dt, coef, ud, work, nsteps)
    step = o.rk104_step if rk == 1 else o.rk3_step
    stages = (10 if rk == 1 else 3) * nsteps
    return host(ud), step(g, co, dt, u0, nsteps), run_scale(g, co, dt, u0, stages)


@pytest.mark.parametrize("wprec", ["fp64", "fp32"])
def test_full_size_paper_run_steps(wprec):
    """The paper's own grid (16384 rho x 64 theta, extremal Kerr, s = -2,
    (l, m) = (2, 0), packet at rho = 1 on the horizon): 3 SSP-RK(3,3) steps,
    every node compared."""
    got, exp_, sc = run_both(I.EXTREMAL_GRAV_HYP, wprec, 3)
    compare(got, exp_, sc, what=f"paper run {wprec}")


def test_hyperboloidal_ssprk104_steps():
    wl = I.EXTREMAL_GRAV_HYP.with_(nr=1500, nth=20)
    got, exp_, sc = run_both(wl, "fp32", 4, rk=1)
    compare(got, exp_, sc, what="hyp ssprk104")


def test_hyperboloidal_handle_against_oracle():
    """Handle path (graph replay, set_gaussian, observe at scri and on the
    horizon) against the oracle over 300 steps of a 600 x 24 run (binary64
    weights: no weight rounding that a last-bit difference could flip)."""
    wl = I.EXTREMAL_GRAV_HYP.with_(nr=600, nth=24)
    p = T.params_from_workload(wl, wprec="fp64")
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, 1.0, wl.a, wl.s, wl.m, 1e-6, "fp64",
               coords=1, S=wl.S)
    co = o.coefficients(g)
    h = T.teuk_create(p)
    coeffs = [0.9 + 0.1j, -0.2 + 0.3j]
    T.teuk_set_gaussian(h, wl.rc, wl.width, coeffs)
    u, _ = T.teuk_get_state(h)
    np.testing.assert_allclose(u, I.gaussian_data(wl, wl.rc, wl.width, coeffs),
                               rtol=0, atol=1e-13)
    _, dt, _ = T.teuk_get_info(h)
    uo = u.copy()
    for _ in range(3):
        T.teuk_step(h, 100)
        uo = o.rk3_step(g, co, dt, uo, 100)
        wave, hor, t = T.teuk_observe(h, wl.S)
        w2, h2 = o.observe(g, uo, wl.S)
        scale = np.max(np.abs(uo))          # the field is still ~0 at scri
        for got, ref in [(wave, w2), (hor, h2)]:
            assert np.max(np.abs(got - ref)) <= 1e-11 * scale, (got, ref)
    assert abs(t - 300 * dt) < 1e-12
