"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: stencils
derived by hand from the paper's printed formulas (tests/golden), polynomial
exactness, convergence orders, the SSP-RK(3,3) stability polynomial, an
independent sympy derivation of the coefficients from Eq. teuk0, the
Regge-Wheeler potential, the spin-weighted harmonic eigenvalue relation, the
paper's printed real matrices M, A, L, and Price's late-time tail.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as o
from paper_2010_04760_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Rounding to the weight formats
# --------------------------------------------------------------------------
def test_round_w_matches_numpy_and_torch():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-9, 5, 2000),
                        [0.0, 65504.0, 65519.9, 65520.0, 2.0 ** -24, 3 * 2.0 ** -26,
                         2.0 ** -25, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11]])
    for v in x:
        assert o.round_w("fp32", v) == float(np.float32(v))
        with np.errstate(over="ignore"):                # overflow to inf is the reference
            ref16 = float(np.float16(v))
        got16 = o.round_w("fp16", v)
        assert got16 == ref16 or (np.isinf(got16) and np.isinf(ref16)), v
    torch = pytest.importorskip("torch")
    xf = x.astype(np.float32).astype(np.float64)      # exactly representable in binary32
    ref = torch.tensor(xf, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([o.round_w("bf16", v) for v in xf])
    np.testing.assert_array_equal(got, ref)


# --------------------------------------------------------------------------
# Tortoise coordinate (Sec. 2.2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("a", [0.0, 0.5, 0.999, 1.0])
def test_tortoise_derivative_and_inverse(a):
    M = 1.0
    rp = M + np.sqrt(max(M * M - a * a, 0.0))
    for r in rp + np.array([0.05, 0.3, 1.0, 4.0, 40.0, 300.0]):
        hstep = 1e-5 * r
        num = (o.rstar_of_r(r + hstep, M, a) - o.rstar_of_r(r - hstep, M, a)) / (2 * hstep)
        exact = (r * r + a * a) / (r * r - 2 * M * r + a * a)
        assert abs(num / exact - 1.0) < 1e-7
        rs = o.rstar_of_r(r, M, a)
        assert abs(o.r_of_rstar(rs, M, a) - r) < 1e-12 * r


def test_tortoise_schwarzschild_lambert_w():
    from scipy.special import lambertw
    for rs in [-60.0, -10.0, 0.0, 3.0, 50.0, 250.0]:
        r_exact = 2.0 * (1.0 + lambertw(np.exp(rs / 2.0 - 1.0)).real)
        assert abs(o.r_of_rstar(rs, 1.0, 0.0) - r_exact) < 1e-12 * r_exact


def test_tortoise_inverse_resolves_r_minus_r_plus_near_the_horizon():
    """Towards the horizon r - r_+ falls off exponentially in r* (Sec. 2.2's
    tortoise relation), below the spacing of binary64 numbers near r_+ by
    r* ~ -70 M at a = 0; the oracle inverts for r - r_+ itself. At a = 0 it is
    2 W(exp(r*/2M - 1)) (Lambert W); for a = 0.7 M and a = M the forward map,
    evaluated at 50 digits at the returned r - r_+, must give r* back."""
    from scipy.special import lambertw
    for rs in [-70.0, -300.0, -1400.0]:
        exact = 2.0 * lambertw(np.exp(rs / 2.0 - 1.0)).real
        assert abs(o.x_of_rstar(rs, 1.0, 0.0) / exact - 1.0) < 1e-12, rs
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for a in (0.7, 1.0):
        rp = 1.0 + np.sqrt(1.0 - a * a)
        for rs in [-40.0, -200.0, -600.0]:
            x = mp.mpf(o.x_of_rstar(rs, 1.0, a))
            if a < 1.0:
                d = mp.sqrt(1 - mp.mpf(a) ** 2)
                mrp, mrm = 1 + d, 1 - d
                back = (mrp + x + (2 * mrp / (mrp - mrm)) * mp.log(x / 2)
                        - (2 * mrm / (mrp - mrm)) * mp.log((x + mrp - mrm) / 2))
            else:
                back = 1 + x + 2 * mp.log(x) - 2 / x
            assert abs(float(back) - rs) < 1e-12 * abs(rs), (a, rs, float(back))
        assert o.r_of_rstar(-40.0, 1.0, a) == rp + o.x_of_rstar(-40.0, 1.0, a)


def test_coefficients_near_the_horizon_keep_their_relative_accuracy():
    """Delta = (r - r_+)(r - r_-) formed from r - r_+: A^thth = Delta/Sigma^2
    and Im C (s m a term aside, proportional to Delta) at r* = -70 M agree
    with a 50-digit evaluation at the same r - r_+ to 1e-13 relative."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for a, s, m in [(0.0, 0, 0), (0.5, -1, 0), (0.999, -2, 2)]:
        g = o.grid(7, 5, -70.0, -64.0, 1.0, a, s, m)
        co = o.coefficients(g)
        ma = mp.mpf(a)
        d = mp.sqrt(1 - ma ** 2)
        for i in range(7):
            x = mp.mpf(o.x_of_rstar(-70.0 + i, 1.0, a))
            r = 1 + d + x
            Delta = x * (x + 2 * d)
            for j in range(5):
                th = mp.mpf((j + 0.5) * np.pi / 5)
                varpi = r * r + ma ** 2
                Sigma2 = varpi ** 2 - ma ** 2 * Delta * mp.sin(th) ** 2
                ath = Delta / Sigma2
                assert abs(co[7, j, i] / float(ath) - 1.0) < 1e-13, (a, i, j)


# --------------------------------------------------------------------------
# WENO5 (Sec. 3.1.2)
# --------------------------------------------------------------------------
def _stencil_from_impulses(dir, length, deriv):
    n = 32
    coeffs = []
    for k in range(length):
        f = np.zeros(n)
        i0 = 12
        off = (-3 if dir > 0 else -2) if deriv else (-2 if dir > 0 else -1)
        f[i0 + off + k] = 1.0
        D = o.weno5_deriv_1d(f, 1.0, dir, periodic=True, force_w=[0.1, 0.6, 0.3],
                             return_wq=False)
        coeffs.append(D[i0] * 60.0)
    return coeffs


def test_linear_weights_reproduce_golden_stencils():
    rows = {r[0]: [int(v) for v in r[1:]] for r in _golden_rows("weno5_linear_stencils.txt")}
    assert np.allclose(_stencil_from_impulses(+1, 6, True), rows["deriv_plus"], atol=1e-12)
    assert np.allclose(_stencil_from_impulses(-1, 6, True), rows["deriv_minus"], atol=1e-12)
    # interface values: f-hat with omega = d over unit impulses
    for dir, key in [(+1, "flux_plus"), (-1, "flux_minus")]:
        got = []
        for k in range(5):
            f5 = np.zeros(5)
            f5[k] = 1.0
            w = np.array([0.1, 0.6, 0.3])
            fl = o._load().orc_weno5_flux(0, dir, o._ptr(f5), 1e-6, o._ptr(w), None, None)
            got.append(fl * 60.0)
        assert np.allclose(got, rows[key], atol=1e-12)


@pytest.mark.parametrize("wprec", ["fp64", "fp32", "fp16", "bf16", "f64r"])
@pytest.mark.parametrize("dir", [1, -1])
def test_linear_data_gives_linear_weights(wprec, dir):
    u = {"fp64": 2.0 ** -53, "f64r": 2.0 ** -53, "fp32": 2.0 ** -24, "fp16": 2.0 ** -11,
         "bf16": 2.0 ** -8}[wprec]
    rng = np.random.default_rng(1)
    for _ in range(50):
        c0, c1 = rng.standard_normal(2) * 10.0 ** rng.integers(-3, 4, 2)
        f5 = c0 + c1 * np.arange(5)
        w = o.weno5_weights(f5, dir, wprec)
        # first differences carry the binary64 cancellation error u64 |f| / |c1|
        tol = 8 * u + 64 * 2.0 ** -53 * (1.0 + np.max(np.abs(f5)) / abs(c1))
        assert np.all(np.abs(w - [0.1, 0.6, 0.3]) <= tol), (w, wprec)


@pytest.mark.parametrize("dir", [1, -1])
def test_linear_scheme_exact_to_degree_five(dir):
    n, h = 40, 0.1
    x = np.arange(n) * h
    for deg in range(6):
        f = (x - 1.3) ** deg
        D = o.weno5_deriv_1d(f, h, dir, periodic=False, force_w=[0.1, 0.6, 0.3])
        ex = deg * (x - 1.3) ** (deg - 1) if deg else 0 * x
        sl = slice(4, n - 4)
        assert np.max(np.abs(D[sl] - ex[sl])) < 1e-9 * max(1, np.max(np.abs(ex[sl])))
    f = (x - 1.3) ** 6
    D = o.weno5_deriv_1d(f, h, dir, periodic=False, force_w=[0.1, 0.6, 0.3])
    assert np.max(np.abs(D[4:n - 4] - 6 * (x[4:n - 4] - 1.3) ** 5)) > 1e-6


@pytest.mark.parametrize("dir", [1, -1])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_each_candidate_stencil_exact_to_degree_three(dir, k):
    n, h = 40, 0.1
    x = np.arange(n) * h
    w = np.zeros(3)
    w[k] = 1.0
    for deg in range(4):
        f = (x - 0.7) ** deg
        D = o.weno5_deriv_1d(f, h, dir, periodic=False, force_w=w)
        ex = deg * (x - 0.7) ** (deg - 1) if deg else 0 * x
        assert np.max(np.abs(D[4:n - 4] - ex[4:n - 4])) < 1e-9
    f = (x - 0.7) ** 4
    D = o.weno5_deriv_1d(f, h, dir, periodic=False, force_w=w)
    assert np.max(np.abs(D[4:n - 4] - 4 * (x[4:n - 4] - 0.7) ** 3)) > 1e-5


def test_smooth_weights_approach_linear_weights_at_second_order():
    devs = []
    for n in (64, 128, 256):
        h = 1.0 / n
        x = np.arange(n) * h
        f = np.sin(2 * np.pi * x)
        _, w, _ = o.weno5_deriv_1d(f, h, 1, periodic=True, return_wq=True)
        xm = x + 0.5 * h
        mask = np.abs(np.cos(2 * np.pi * xm)) > 0.3            # away from critical points
        devs.append(np.max(np.abs(w[mask] - [0.1, 0.6, 0.3])))
    orders = np.log2(np.array(devs[:-1]) / np.array(devs[1:]))
    assert np.all(orders > 1.8), (devs, orders)


@pytest.mark.parametrize("dir", [1, -1])
def test_fifth_order_convergence_on_periodic_advection(dir):
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        x = np.arange(n) * h
        T = 0.25
        ns = int(np.ceil(T / (0.4 * h ** (5.0 / 3.0))))
        f = o.advect_1d(np.sin(2 * np.pi * x), h, T / ns, ns, dir=dir)
        errs.append(np.mean(np.abs(f - np.sin(2 * np.pi * (x - dir * T)))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.7), orders


@pytest.mark.parametrize("wprec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dir", [1, -1])
def test_reduced_weights_within_rounding_of_fp64_weights(wprec, dir):
    """The reduced-precision reading differs from the paper's binary64 weights
    by a few units of the weight format's rounding, at every scale; the flux
    difference obeys |fhat_W - fhat_64| <= sum_k |dw_k| |q_k - q_1|."""
    u = {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[wprec]
    rng = np.random.default_rng(7)
    worst = 0.0
    for trial in range(3000):
        scale = 10.0 ** rng.uniform(-12, 8)
        f5 = rng.standard_normal(5) * scale
        if trial % 3 == 0:                       # smooth-ish stencils
            f5 = scale * (rng.standard_normal() + rng.standard_normal() * np.arange(5)
                          + 0.01 * rng.standard_normal(5))
        w64 = o.weno5_weights(f5, dir, "fp64")
        wW = o.weno5_weights(f5, dir, wprec)
        dw = np.abs(wW - w64)
        worst = max(worst, np.max(dw) / u)
        lib = o._load()
        wo, qo = np.zeros(3), np.zeros(3)
        fW = lib.orc_weno5_flux(o.WPREC[wprec], dir, o._ptr(f5), 1e-6, None, o._ptr(wo), o._ptr(qo))
        f64 = lib.orc_weno5_flux(0, dir, o._ptr(f5), 1e-6, None, None, None)
        bound = np.sum(np.abs(wo - w64) * np.abs(qo - qo[1])) + 1e-13 * np.max(np.abs(f5))
        assert abs(fW - f64) <= bound, (f5, fW, f64, bound)
        # the promoted weights sum to one in binary64 (Sec. 3.1.3)
        assert abs((wo[0] + wo[1]) + wo[2] - 1.0) <= 2.0 ** -52, wo
    assert worst < 12.0, worst


def test_reduced_reading_in_binary64_equals_paper_formula():
    rng = np.random.default_rng(11)
    for dir in (1, -1):
        for _ in range(2000):
            f5 = rng.standard_normal(5) * 10.0 ** rng.uniform(-10, 6)
            assert np.max(np.abs(o.weno5_weights(f5, dir, "f64r")
                                 - o.weno5_weights(f5, dir, "fp64"))) < 1e-13


# --------------------------------------------------------------------------
# SSP-RK(3,3) (Sec. 3.2)
# --------------------------------------------------------------------------
def test_ssprk33_stability_polynomial():
    c = [float(Fraction(v)) for v in _golden_rows("ssprk33_stability.txt")[0]]
    for z in [0.3, -1.2, 0.7j, -0.4 + 1.1j, 2.0 - 0.5j]:
        R = sum(ck * z ** k for k, ck in enumerate(c))
        assert abs(o.rk3_linear(z, 1.0, 1) - R) < 1e-14 * max(1, abs(R))


def test_ssprk33_third_order():
    lam = -0.8 + 2.0j
    errs = []
    for ns in (20, 40, 80):
        errs.append(abs(o.rk3_linear(lam, 1.0 / ns, ns) - np.exp(lam)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 3.0) < 0.15), orders


# --------------------------------------------------------------------------
# SSP coefficients stated in Sec. 3.2: C = 1 for SSP-RK(3,3), C = 6 for
# SSP-RK(10,4). The one-step polynomial R(z) is recovered from the oracle's
# integrators at roots of unity; C is the largest value for which R(-C + w)
# has no negative Taylor coefficient in w (absolute monotonicity on [-C, 0]).
# --------------------------------------------------------------------------
def _stability_poly(step, degree, radius):
    # sampled on a circle of the method's radius so that the small high-order
    # coefficients are recovered with small relative error
    n = 32
    zs = radius * np.exp(2j * np.pi * np.arange(n) / n)
    vals = np.array([step(z, 1.0, 1) for z in zs])
    c = np.array([np.mean(vals * zs ** (-m)) for m in range(n)])
    assert np.max(np.abs(c[degree + 1:]) * radius ** np.arange(degree + 1, n)) < 1e-10
    return np.real(c[:degree + 1])


def _shifted_coeffs(c, C):
    """Coefficients of R(-C + w) in w, and the size of the terms summed for
    each (the round-off scale of the expansion)."""
    from math import comb
    deg = len(c) - 1
    val = np.array([sum(c[k] * comb(k, m) * (-C) ** (k - m) for k in range(m, deg + 1))
                    for m in range(deg + 1)])
    size = np.array([sum(abs(c[k]) * comb(k, m) * C ** (k - m) for k in range(m, deg + 1))
                     for m in range(deg + 1)])
    return val, size


@pytest.mark.parametrize("step,degree,order,C", [(o.rk3_linear, 3, 3, 1.0),
                                                 (o.rk104_linear, 10, 4, 6.0)])
def test_ssp_coefficient_and_order(step, degree, order, C):
    from math import factorial
    c = _stability_poly(step, degree, C)
    for k in range(order + 1):
        assert abs(c[k] - 1.0 / factorial(k)) < 1e-12
    if degree > order:                                   # exactly this order
        assert abs(c[order + 1] - 1.0 / factorial(order + 1)) > 1e-5
    val, size = _shifted_coeffs(c, C)
    assert np.all(val >= -1e-12 * size), val
    val, size = _shifted_coeffs(c, C * 1.02)
    assert np.min(val + 1e-12 * size) < 0.0              # C is the threshold


def test_ssprk104_fourth_order_convergence():
    lam = -0.8 + 2.0j
    errs = [abs(o.rk104_linear(lam, 1.0 / ns, ns) - np.exp(lam)) for ns in (10, 20, 40)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 4.0) < 0.2), orders


# --------------------------------------------------------------------------
# FD6 + KO8 comparison scheme (Sec. 3.1.1)
# --------------------------------------------------------------------------
def test_fd6_exact_to_degree_six_and_sixth_order():
    n, h = 48, 0.1
    x = np.arange(n) * h
    for deg in range(7):
        f = (x - 2.1) ** deg
        D, _ = o.fd6_ko8_1d(f, h, 0.01, periodic=False)
        ex = deg * (x - 2.1) ** (deg - 1) if deg else 0 * x
        assert np.max(np.abs(D[5:n - 5] - ex[5:n - 5])) < 1e-8 * max(1, np.max(np.abs(ex)))
    f = (x - 2.1) ** 7
    D, _ = o.fd6_ko8_1d(f, h, 0.01, periodic=False)
    assert np.max(np.abs(D[5:n - 5] - 7 * (x[5:n - 5] - 2.1) ** 6)) > 1e-6
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        x = np.arange(n) * h
        D, _ = o.fd6_ko8_1d(np.sin(2 * np.pi * x), h, 0.01)
        errs.append(np.max(np.abs(D - 2 * np.pi * np.cos(2 * np.pi * x))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 5.8), orders


def test_ko8_annihilates_degree_seven_and_has_its_fourier_symbol():
    n, h, sigma = 48, 0.1, 0.37
    x = np.arange(n) * h
    for deg in range(8):
        _, Q = o.fd6_ko8_1d((x - 2.1) ** deg, h, sigma, periodic=False)
        assert np.max(np.abs(Q[5:n - 5])) < 1e-9
    n = 64
    h = 1.0 / n
    x = np.arange(n) * h
    for k in (1, 5, 16, 31):
        f = np.cos(2 * np.pi * k * x + 0.3)
        _, Q = o.fd6_ko8_1d(f, h, sigma)
        symbol = sigma * (2.0 * np.sin(np.pi * k * h)) ** 8 / (256.0 * h)
        assert np.max(np.abs(Q - symbol * f)) < 1e-12 * max(1.0, symbol)


@pytest.mark.parametrize("wprec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("coords", [0, 1])
def test_weno_operator_homogeneous_with_scaled_eps(wprec, coords):
    """WENO5's weights (Sec. 3.1.2) depend on the data through eps + IS_k,
    and IS_k is quadratic in the data, so scaling the data by 4 and eps by 16
    scales every eps + IS_k by 16 and leaves the weights unchanged; the
    reduced-precision reading scales the differences to a power of two first
    (Sec. 3.1.3), which absorbs the 4 exactly. The rest of the right-hand side
    is linear, so F_16eps(4u) = 4 F_eps(u), and in binary floating point bit
    for bit (powers of two commute with every rounding): the identity the
    CUDA step's scaled second stage rests on. Multi-scale data, both
    coordinate systems, both theta schemes."""
    for theta_mode in (0, 1):
        wl = (I.KERR_GRAV.with_(nr=96, nth=10) if coords == 0
              else I.EXTREMAL_GRAV_HYP.with_(nr=120, nth=8))
        args = (wl.nr, wl.nth, wl.rs_min, wl.rs_max, wl.M, wl.a, wl.s, wl.m)
        g1 = o.grid(*args, eps=wl.eps, wprec=wprec, theta_mode=theta_mode, coords=wl.coords,
                    S=wl.S)
        g16 = o.grid(*args, eps=16.0 * wl.eps, wprec=wprec, theta_mode=theta_mode,
                     coords=wl.coords, S=wl.S)
        co = o.coefficients(g1)
        u = I.multiscale_state(wl.nr, wl.nth, 21)
        np.testing.assert_array_equal(o.rhs(g16, co, 4.0 * u), 4.0 * o.rhs(g1, co, u))
        # and eps matters: unscaled eps on the scaled data changes the weights
        assert np.any(o.rhs(g1, co, 4.0 * u) != 4.0 * o.rhs(g1, co, u))

