"""Pins of the extended-precision oracle (oracle/teuk_oracle_ld.c), which
carries the state, weights and fluxes in C long double to measure the binary64
state's own round-off (the paper's quad-precision baseline, Sec. 2.3 on
high-precision numerics and Sec. 3.1.3).

It is tied to the mathematics and to the binary64 oracle, not to itself:
  - its precision: on data linear in the grid index every WENO5 candidate
    value equals the interface value and the weights sum to one, so the flux
    and the radial derivative are known in closed form (Sec. 3.1.2); the
    extended oracle reproduces them, and the whole right-hand side of such a
    state, to a few units of the long double format, a bound binary64
    arithmetic misses by orders of magnitude (checked on the binary64 oracle);
  - its formula: on generic data (smooth, multi-scale, both coordinate
    systems, both pole parities) its right-hand side agrees with the binary64
    oracle, whose pins tie it to the paper, within the per-node round-off
    scale of binary64; so does an evolution of 20 SSP-RK(3,3) steps.
The mistakes planted in tests/test_oracle_mutants.py (the extended list) fail
these pins."""
import numpy as np
import pytest

import oracle as o
from paper_2010_04760_gb300 import inputs as I
from _local_scale import assert_local, rhs_scale, run_scale

L = np.longdouble
EPS_LD = float(np.finfo(np.longdouble).eps)
EPS_D = float(np.finfo(np.float64).eps)


def test_extended_format_is_wider_than_binary64():
    assert o.ld_mant_dig() >= 64
    assert np.finfo(np.longdouble).nmant + 1 == o.ld_mant_dig()
    assert EPS_LD * 2048 <= EPS_D


@pytest.mark.parametrize("dir,at", [(+1, 2.5), (-1, 1.5)])
def test_flux_of_linear_data_in_closed_form(dir, at):
    """f_k = a + b k: every candidate stencil gives a + b (k of the interface),
    whatever the weights (they sum to one), for any eps."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(50):
        a = L(rng.uniform(-2, 2)) / L(3)
        b = L(rng.uniform(-2, 2)) / L(7)
        f = np.array([a + b * L(k) for k in range(5)], dtype=L)
        ex = a + b * L(at)
        for eps in (1e-6, 1e-40, 1.0):
            got = o.ld_weno5_flux(f, dir, eps)
            scale = float(np.max(np.abs(f)))
            worst = max(worst, float(abs(got - ex)) / scale)
    assert worst <= 16 * EPS_LD


def _linear_state(nr, nth, seed):
    """Each component a + b i (i the radial index), the same in every row."""
    rng = np.random.default_rng(seed)
    i = np.arange(nr, dtype=L)
    u = np.empty((4, nth, nr), dtype=L)
    ab = []
    for c in range(4):
        a = L(rng.uniform(-1, 1)) / L(3)
        b = L(rng.uniform(-1, 1)) / L(7 * nr)
        u[c] = (a + b * i)[None, :]
        ab.append((a, b))
    return u, ab


def _closed_form_rhs(g, co, ab):
    """F of the linear state away from the radial edges: D = b / h exactly
    and the theta differences of equal rows vanish (parity +1)."""
    nr, nth = g.nr, g.nth
    h = L((g.rs_max - g.rs_min) / (nr - 1))          # the binary64 spacing
    i = np.arange(nr, dtype=L)
    c = co.astype(L)
    j1 = np.clongdouble(1j)
    val = [np.broadcast_to((a + b * i)[None, :], (nth, nr)) for a, b in ab]
    D = [b / h for _, b in ab]
    psi = val[0] + j1 * val[1]
    pi = val[2] + j1 * val[3]
    Dpsi = D[0] + j1 * D[1]
    Dpi = D[2] + j1 * D[3]
    K = c[1] + j1 * c[2]
    Bt = c[3] + j1 * c[4]
    C = c[5] + j1 * c[6]
    Fpsi = pi - c[0] * Dpsi
    Fpi = c[9] * Dpi + K * Dpsi + Bt * pi + C * psi
    F = np.stack([Fpsi.real, Fpsi.imag, Fpi.real, Fpi.imag]).astype(L)
    R = max(float(np.max(np.abs(v))) for v in val)
    dth = np.pi / nth
    ca = np.abs(co.astype(np.float64))
    S = ((ca[0] + ca[9] + ca[1] + ca[2]) * R / float(h) + (ca[3] + ca[4] + ca[5] + ca[6] + 1) * R
         + (ca[7] * 64 / (12 * dth ** 2) + ca[8] * 18 / (12 * dth)) * R)
    return F, np.broadcast_to(S, F.shape)


@pytest.mark.parametrize("a,s,m,coords", [(0.9, -2, 2, 0), (0.0, 0, 0, 0), (0.5, -1, 1, 0),
                                          (1.0, -2, 0, 1), (0.7, 0, 2, 1)])
def test_rhs_of_linear_state_in_closed_form(a, s, m, coords):
    """The extended right-hand side of a row-constant state linear in the
    radial index (r*, or rho on the hyperboloidal slices, whose pi rows move
    with their own speed c) matches its closed form to 8 units of the long
    double format of the terms' size at nodes whose stencils stay inside the
    grid; the binary64 oracle on the same state (rounded to binary64) does
    not."""
    if coords == 1:
        rho_p = o.horizon_rho(1.0, a, 20.0)
        g = o.grid(96, 6, rho_p + 0.5, 15.0, 1.0, a, s, m, coords=1, S=20.0)
    else:
        g = o.grid(96, 6, -30.0, 60.0, 1.0, a, s, m)
    co = o.coefficients(g)
    u, ab = _linear_state(g.nr, g.nth, seed=11)
    ex, S = _closed_form_rhs(g, co, ab)
    got = o.ld_rhs(g, co, u)
    inner = slice(3, g.nr - 3)
    err = np.abs((got - ex)[..., inner]).astype(np.float64)
    bound = 8 * EPS_LD * S[..., inner]
    assert np.all(err <= bound), float(np.max(err / bound))
    # the same bound is beyond binary64 arithmetic
    got_d = o.rhs(g, co, u.astype(np.float64))
    err_d = np.abs((got_d.astype(L) - ex)[..., inner]).astype(np.float64)
    assert np.max(err_d / bound) > 64


CASES = [
    # (label, workload, state maker)
    ("kerr s=-2 m=2 (parity +1)", I.KERR_GRAV.with_(nr=160, nth=12), "smooth"),
    ("kerr s=-1 m=2 (parity -1)", I.KERR_GRAV.with_(nr=150, nth=9, s=-1, a=0.6), "smooth"),
    ("kerr multiscale", I.KERR_GRAV.with_(nr=128, nth=10), "multiscale"),
    ("hyperboloidal extremal", I.EXTREMAL_GRAV_HYP.with_(nr=300, nth=8), "smooth"),
    ("hyperboloidal multiscale", I.EXTREMAL_GRAV_HYP.with_(nr=200, nth=8, m=1), "multiscale"),
]


def _grid(wl):
    return o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, wl.M, wl.a, wl.s, wl.m, wl.eps, "fp64",
                  coords=wl.coords, S=wl.S)


def _state(wl, kind, seed=5):
    if kind == "multiscale":
        return I.multiscale_state(wl.nr, wl.nth, seed)
    return I.random_state(wl.nr, wl.nth, seed)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rhs_agrees_with_binary64_oracle(case):
    label, wl, kind = CASES[case]
    g = _grid(wl)
    co = o.coefficients(g)
    u = _state(wl, kind)
    F_d = o.rhs(g, co, u)
    F_l = o.ld_rhs(g, co, u.astype(L))
    assert_local(F_l.astype(np.float64), F_d, rhs_scale(g, co, u), what=label)


@pytest.mark.parametrize("case", [0, 1, 3])
def test_evolution_agrees_with_binary64_oracle(case):
    """20 SSP-RK(3,3) steps: the two evolutions differ by binary64 round-off
    only (and do differ: the extended one is not the binary64 code)."""
    label, wl, kind = CASES[case]
    g = _grid(wl)
    co = o.coefficients(g)
    u = _state(wl, kind)
    h = (wl.rs_max - wl.rs_min) / (wl.nr - 1)
    dt = 0.2 * h / max(float(np.max(np.abs(co[0]))), float(np.max(np.abs(co[9]))), 1e-3)
    dt = min(dt, 0.02)
    u_d = o.rk3_step(g, co, dt, u, 20)
    u_l = o.ld_rk3_step(g, co, dt, u.astype(L), 20)
    assert_local(u_l.astype(np.float64), u_d, run_scale(g, co, dt, u, 60), what=label)
    assert np.any(u_l != u_d.astype(L))


def test_unsupported_schemes_are_refused():
    g = o.grid(32, 4, -10.0, 10.0, theta_mode=1)
    with pytest.raises(ValueError):
        o.ld_rhs(g, np.zeros((10, 4, 32)), np.zeros((4, 4, 32)))
    g = o.grid(32, 4, -10.0, 10.0, scheme=1)
    with pytest.raises(ValueError):
        o.ld_rk3_step(g, np.zeros((10, 4, 32)), 0.1, np.zeros((4, 4, 32)))


@pytest.mark.parametrize("case", [0, 3])
def test_evolution_carries_the_extended_precision(case):
    """A perturbation of 256 units of the long double format at one node
    (an eighth of a binary64 unit, which binary64 arithmetic would round
    away) survives three SSP-RK(3,3) steps at CFL 0.01 at that node: every
    stage and every combination keeps the extra bits."""
    label, wl, kind = CASES[case]
    g = _grid(wl)
    co = o.coefficients(g)
    u = I.random_state(wl.nr, wl.nth, 3).astype(L)
    c, j, i = 2, wl.nth // 2, wl.nr // 2
    u[c, j, i] = L(0.75)
    delta = L(256) * np.spacing(u[c, j, i])
    assert float(delta) < float(np.spacing(np.float64(0.75))) / 4
    h = (wl.rs_max - wl.rs_min) / (wl.nr - 1)
    dt = 0.01 * h / max(float(np.max(np.abs(co[0]))), float(np.max(np.abs(co[9]))), 1e-3)
    base = o.ld_rk3_step(g, co, dt, u, 3)
    up = u.copy()
    up[c, j, i] += delta
    pert = o.ld_rk3_step(g, co, dt, up, 3)
    ratio = float((pert[c, j, i] - base[c, j, i]) / delta)
    assert 0.8 <= ratio <= 1.2, (label, ratio)
