"""Physics pins of the CPU oracle: coefficients against an independent sympy
derivation from Eq. teuk0, the Regge-Wheeler potential, the spin-weighted
harmonic eigenvalue relation, the paper's printed real matrices M, A, L
(Eqs. m_matrix, a_matrix, l_matrix) and Price's t^-3 tail."""
import os

import numpy as np
import pytest

import oracle as o
from paper_2010_04760_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sympy_coefficients():
    """Second-order normalised coefficients of Eq. teuk0 after the ingoing
    azimuth phi~ = phi + int a/Delta dr and tortoise r*, derived here with a
    symbolic chain rule (no formula is copied from the oracle)."""
    sp = pytest.importorskip("sympy")
    r, th = sp.symbols("r theta", positive=True)
    M, a, s, m = sp.symbols("M a s m", real=True)
    f0, fx, fxx, ft, ftt, fth, fthth, ftx = sp.symbols("f0 fx fxx ft ftt fth fthth ftx")
    varpi = r ** 2 + a ** 2
    Delta = r ** 2 - 2 * M * r + a ** 2
    dxdr = varpi / Delta
    chain = {f0: dxdr * fx, fx: dxdr * fxx, ft: dxdr * ftx}

    def Dr(E):      # d/dr of exp(i m int a/Delta) * E, divided by that factor
        out = sp.diff(E, r) + sp.I * m * a / Delta * E
        for sym, d in chain.items():
            out += sp.diff(E, sym) * d
        return out

    def Dth(E):
        return sp.diff(E, th) + sp.diff(E, f0) * fth + sp.diff(E, fth) * fthth

    sn, cs = sp.sin(th), sp.cos(th)
    radial = Delta ** (-s) * Dr(Delta ** (s + 1) * Dr(f0))
    angular = Dth(sn * Dth(f0)) / sn
    E = (-(varpi ** 2 / Delta - a ** 2 * sn ** 2) * ftt
         - 4 * M * a * r / Delta * (sp.I * m) * ft
         - 2 * s * (r - M * (r ** 2 - a ** 2) / Delta + sp.I * a * cs) * ft
         + radial + angular
         + (1 / sn ** 2 - a ** 2 / Delta) * (-m ** 2) * f0
         + 2 * s * (a * (r - M) / Delta + sp.I * cs / sn ** 2) * (sp.I * m) * f0
         - (s ** 2 * cs ** 2 / sn ** 2 - s) * f0)
    E = sp.expand(E)
    ctt = sp.diff(E, ftt)
    coef = {k: -sp.diff(E, v) / ctt for k, v in
            [("Axx", fxx), ("Bx", fx), ("Ath", fthth), ("Bth", fth), ("Bt", ft),
             ("C", f0), ("Atx", ftx)]}
    b = sp.sqrt(coef["Axx"])
    bstar = (Delta / varpi) * sp.diff(b, r)
    K = coef["Bx"] - b * bstar - b * coef["Bt"]
    args = (r, th, M, a, s, m)
    fn = {k: sp.lambdify(args, v, "numpy") for k, v in coef.items()}
    fn["b"] = sp.lambdify(args, b, "numpy")
    fn["K"] = sp.lambdify(args, K, "numpy")
    return fn


@pytest.fixture(scope="module")
def symcoef():
    return _sympy_coefficients()


@pytest.mark.parametrize("a,s,m", [(0.0, 0, 0), (0.999, -2, 2), (1.0, 0, 0),
                                   (0.5, -1, 3), (0.3, 2, -1), (0.8, -2, 0)])
def test_coefficients_match_symbolic_derivation(symcoef, a, s, m):
    M = 1.0
    rp = M + np.sqrt(max(M * M - a * a, 0.0))
    rng = np.random.default_rng(3)
    for _ in range(20):
        r = rp + 10.0 ** rng.uniform(-1.5, 2.5)
        th = rng.uniform(0.05, np.pi - 0.05)
        got = o.coeff_point(r, th, M, a, s, m)
        args = (r, th, M, a, s, m)
        exp_ = [complex(symcoef["b"](*args)), complex(symcoef["K"](*args)),
                complex(symcoef["Bt"](*args)), complex(symcoef["C"](*args)),
                complex(symcoef["Ath"](*args)), complex(symcoef["Bth"](*args))]
        gotc = [got[0], got[1] + 1j * got[2], got[3] + 1j * got[4], got[5] + 1j * got[6],
                got[7], got[8]]
        for e, g in zip(exp_, gotc):
            assert abs(e - g) <= 1e-10 * max(1.0, abs(e)), (a, s, m, r, th, e, g)
        assert abs(complex(symcoef["Atx"](*args))) < 1e-12      # no t-r* cross term


@pytest.mark.parametrize("ell", [0, 1, 2, 5])
def test_schwarzschild_scalar_reduces_to_regge_wheeler(ell):
    """a = s = m = 0: with psi = u / r the r* equation becomes
    u_tt = u_** - V u, V = (1 - 2M/r)(l(l+1)/r^2 + 2M/r^3)."""
    M = 1.0
    for r in [2.1, 3.0, 6.0, 20.0, 150.0]:
        c = o.coeff_point(r, 1.1, M, 0.0, 0, 0)
        b, K, Ath = c[0], c[1], c[7]
        assert abs(b - 1.0) < 1e-14 and abs(c[2]) + abs(c[3]) + abs(c[4]) + abs(c[5]) + abs(c[6]) < 1e-14
        Delta = r * r - 2 * M * r
        rp = Delta / r ** 2                                     # dr/dr*
        rpp = rp * (2 * (r - M) / r ** 2 - 2 * Delta / r ** 3)  # d2r/dr*2
        coef_up = -2 * rp / r ** 2 + K / r                      # multiplies u'
        coef_u = -rpp / r ** 2 + 2 * rp ** 2 / r ** 3 - K * rp / r ** 2 - ell * (ell + 1) * Ath / r
        V = (1 - 2 * M / r) * (ell * (ell + 1) / r ** 2 + 2 * M / r ** 3)
        assert abs(coef_up) < 1e-14 * (1 + abs(K / r))
        assert abs(coef_u + V / r) < 1e-12 * max(V / r, 1e-300) + 1e-15


def _eigen_cases():
    rows = []
    with open(os.path.join(GOLDEN, "swsh_eigenvalues.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("case", _eigen_cases())
@pytest.mark.parametrize("a", [0.0, 0.6])
def test_theta_operator_on_spin_weighted_harmonics(case, a):
    """F_pi of (Psi = sY_lm(theta), constant in r*, pi = 0) is
    (Delta/Sigma^2) lambda Psi + i 4 s m a (r-M)/Sigma^2 Psi; the discrete
    operator converges to it at fourth order (3.3+ in L2 when the pole parity
    is odd)."""
    s, l, m, lam = case
    assert lam == -(l - s) * (l + s + 1)
    errs = []
    for nth in (32, 64, 128):
        g = o.grid(16, nth, -10.0, 10.0, 1.0, a, s, m)
        co = o.coefficients(g)
        Y = I.swsh(s, l, m, I.theta_nodes(nth))
        u = np.zeros((4, nth, 16))
        u[0] = Y[:, None]
        F = o.rhs(g, co, u)
        res = F[2][:, 8] / co[7][:, 8] - lam * Y
        errs.append(np.sqrt(np.mean(res ** 2)))
        np.testing.assert_allclose(F[3][:, 8], co[6][:, 8] * Y, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(F[0], 0.0, atol=1e-15)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 3.3), (errs, orders)
    assert errs[-1] < 1e-4 * abs(lam) + 1e-9


@pytest.mark.parametrize("case", _eigen_cases())
@pytest.mark.parametrize("a", [0.0, 0.6])
def test_theta_weno_option_on_spin_weighted_harmonics(case, a):
    """theta_mode 1 (WENO5 first theta derivative, reading): the discrete
    operator still converges to the sY_lm eigenvalue relation (order > 3.3
    over the last refinements once the weights have settled)."""
    s, l, m, lam = case
    errs = []
    for nth in (64, 128, 256):
        g = o.grid(16, nth, -10.0, 10.0, 1.0, a, s, m, 1e-6, "fp64", 1)
        co = o.coefficients(g)
        Y = I.swsh(s, l, m, I.theta_nodes(nth))
        u = np.zeros((4, nth, 16))
        u[0] = Y[:, None]
        F = o.rhs(g, co, u)
        res = F[2][:, 8] / co[7][:, 8] - lam * Y
        errs.append(np.sqrt(np.mean(res ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 3.3, (errs, orders)
    assert errs[-1] < 1e-5 * abs(lam) + 1e-9


def test_theta_weno_stencil_lies_upwind():
    """theta_mode 1 upwinds the Bth dPsi/dtheta term by the sign of its speed
    -Bth (reading): Bth = Delta cot(theta)/Sigma^2 is positive in the
    northern hemisphere, so there the derivative at row j uses the
    negative-direction stencils (rows j-2 .. j+3) and row j-3 cannot enter
    F_pi(j); in the southern hemisphere it is the mirror image (rows
    j-3 .. j+2, row j+3 cannot enter). Rows j +- 3 enter only through this
    derivative (the centred second difference spans j +- 2)."""
    nr, nth = 12, 24
    g = o.grid(nr, nth, -10.0, 10.0, 1.0, 0.6, 0, 0, 1e-6, "fp64", 1)
    co = o.coefficients(g)
    th = I.theta_nodes(nth)
    rng = np.random.default_rng(5)
    u = np.zeros((4, nth, nr))
    u[0] = np.cos(th)[:, None] * (1.0 + 0.1 * rng.standard_normal(nr))[None, :]
    u[1] = np.sin(2 * th)[:, None] * 0.5
    F = o.rhs(g, co, u)
    for j, quiet, loud in [(6, 3, 9), (nth - 1 - 6, nth - 1 - 3, nth - 1 - 9)]:
        assert (co[8][j] > 0).all() == (j < nth // 2)
        for row, moves in [(quiet, False), (loud, True)]:
            v = u.copy()
            v[0][row] += 0.3
            v[1][row] -= 0.2
            dF = np.abs(o.rhs(g, co, v)[2:4, j] - F[2:4, j])
            assert (dF.max() > 1e-6) == moves, (j, row, dF.max())


@pytest.mark.parametrize("scheme,coords", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_assembly_matches_printed_real_matrices(scheme, coords):
    """F = -(M du/dx + L u + A u) with M, A, L exactly as printed in Sec. 2.3,
    using m31 = -Re K, m32 = Im K, a31 = -Re C, a32 = Im C, a33 = -Re Bt,
    a34 = Im Bt, l31 = -(Ath d2/dth2 + Bth d/dth), on data linear in x = r*
    or rho (where every WENO derivative is exact, the hyperboloidal grid's
    extrapolated ghosts included) times sY_lm(theta). On the hyperboloidal
    slices the pi rows' diagonal entry is -c, c = Atr + b (-b when Atr = 0)."""
    s, l, m, a, M = -2, 3, 2, 0.7, 1.0
    nr, nth = 64, 128
    x0, x1 = (5.0, 15.0) if coords == 0 else (2.5, 20.0)
    g = o.grid(nr, nth, x0, x1, M, a, s, m, scheme=scheme, coords=coords, S=20.0)
    co = o.coefficients(g)
    rs = I.rstar_nodes(nr, x0, x1)
    th = I.theta_nodes(nth)
    Y = I.swsh(s, l, m, th)[:, None]
    al, be, ga, de = 0.3 - 0.2j, 0.7 + 0.4j, -0.5 + 0.1j, 0.2 - 0.9j
    psi = (al + be * rs)[None, :] * Y
    pi = (ga + de * rs)[None, :] * Y
    u = np.stack([psi.real, psi.imag, pi.real, pi.imag])
    F = o.rhs(g, co, u)
    du = np.stack([(be * Y).real + 0 * rs, (be * Y).imag + 0 * rs,
                   (de * Y).real + 0 * rs, (de * Y).imag + 0 * rs])
    b, Kr, Ki, Btr, Bti, Cr, Ci, Ath, Bth, c = co
    if coords == 0:
        np.testing.assert_array_equal(c, b)
    lam = -(l - s) * (l + s + 1)
    cth = np.cos(th)[:, None]
    sth = np.sin(th)[:, None]
    ang = lam - s + (m + s * cth) ** 2 / sth ** 2        # (d2 + cot d) Y / Y
    Lpsi = -(Ath * ang) * u[0:2]                          # l31 acting on Psi_R, Psi_I
    m31, m32, a31, a32, a33, a34 = -Kr, Ki, -Cr, Ci, -Btr, Bti
    z = np.zeros_like(b)
    Mm = [[b, z, z, z], [z, b, z, z], [m31, m32, -c, z], [-m32, m31, z, -c]]
    Am = [[z, z, -1 + z, z], [z, z, z, -1 + z], [a31, a32, a33, a34], [-a32, a31, -a34, a33]]
    exp_ = np.zeros_like(u)
    for row in range(4):
        acc = sum(Mm[row][c] * du[c] + Am[row][c] * u[c] for c in range(4))
        if row >= 2:
            acc = acc + Lpsi[row - 2]
        exp_[row] = -acc
    sl = (slice(None), slice(5, nr - 5) if coords == 0 else slice(None))
    for row in range(4):
        scale = np.max(np.abs(exp_[row][sl]))
        err = np.max(np.abs(F[row][sl] - exp_[row][sl]))
        assert err < (1e-12 if row < 2 else 2e-4) * scale, (row, err, scale)


def test_kreiss_oliger_term_damps_in_the_right_hand_side():
    """Sec. 3.1.1 leaves the sign of Q = sigma h^7 D+^4 D-^4 / 256 in the
    evolution open; the damping reading subtracts it. On the sawtooth
    (-1)^i, D+ D- multiplies by -4/h^2, so Q = (sigma/h) u and the scheme's
    right-hand side must change by exactly -(sigma/h) u (in every component,
    away from the ghost-affected edges) when sigma is switched on."""
    nr, nth, sigma = 40, 6, 0.3
    x0, x1 = -20.0, 40.0
    h = (x1 - x0) / (nr - 1)
    saw = (-1.0) ** np.arange(nr)
    for comp in range(4):
        u = np.zeros((4, nth, nr))
        u[comp] = saw[None, :]
        F = {}
        for sg in (0.0, sigma):
            g = o.grid(nr, nth, x0, x1, 1.0, 0.0, 0, 0, scheme=1, ko_sigma=sg)
            F[sg] = o.rhs(g, o.coefficients(g), u)
        diff = (F[sigma] - F[0.0])[:, :, 5:nr - 5]
        want = np.zeros_like(diff)
        want[comp] = -(sigma / h) * saw[None, 5:nr - 5]
        np.testing.assert_allclose(diff, want, rtol=0, atol=1e-9 * sigma / h)


def test_constant_scalar_state_is_stationary():
    for a in (0.0, 0.9):
        g = o.grid(40, 12, -20.0, 40.0, 1.0, a, 0, 0)
        co = o.coefficients(g)
        u = np.zeros((4, 12, 40))
        u[0] = 0.37
        u[1] = -1.2
        np.testing.assert_allclose(o.rhs(g, co, u), 0.0, atol=1e-14)


def test_observe_gathers_nodes_and_one_sided_derivative():
    g = o.grid(50, 6, -10.0, 39.0, 1.0, 0.0, 0, 0)
    rs = I.rstar_nodes(50, -10.0, 39.0)
    u = np.zeros((4, 6, 50))
    for c in range(4):
        u[c] = (c + 1) * (rs ** 2)[None, :] + np.arange(6)[:, None]
    wave, hor = o.observe(g, u, 20.4)
    np.testing.assert_array_equal(wave[:, 0], u[0][:, 30])
    np.testing.assert_array_equal(o.observe(g, u, 20.6)[0][:, 1], u[1][:, 31])   # nearest node
    np.testing.assert_array_equal(o.observe(g, u, -30.0)[0][:, 0], u[0][:, 0])   # clamped
    np.testing.assert_array_equal(o.observe(g, u, 99.0)[0][:, 0], u[0][:, 49])
    np.testing.assert_array_equal(hor[:, 2], u[2][:, 0])
    np.testing.assert_allclose(hor[:, 4], 2 * rs[0] * 1, rtol=1e-12)
    np.testing.assert_allclose(hor[:, 5], 2 * rs[0] * 2, rtol=1e-12)


@pytest.mark.slow
def test_price_tail_exponent_schwarzschild_l0():
    """s = m = a = 0, l = 0 data: the local index p = t dPsi/dt / Psi at fixed
    r* tends to -(2l+3) = -3 (Sec. 3 on late-time tails; p as in Sec. 4)."""
    L, h, T = 400.0, 0.5, 650.0
    nr, nth = int(round(2 * L / h)) + 1, 6
    g = o.grid(nr, nth, -L, L, 1.0, 0.0, 0, 0)
    co = o.coefficients(g)
    w = I.Workload(name="tail", nr=nr, nth=nth, rs_min=-L, rs_max=L, rc=0.0,
                   width=4.0, ells=(0,), seed=0)
    u = I.initial_data(w)
    dt = 0.4 * h
    chunk = int(round(10.0 / dt))
    ie = int(round((20.0 + L) / h))
    ts, ps = [], []
    t = 0.0
    while t < T:
        u = o.rk3_step(g, co, dt, u, chunk)
        t += chunk * dt
        ts.append(t)
        ps.append(u[0, 0, ie])
    ts, ps = np.array(ts), np.array(ps)
    p = ts[1:-1] * (ps[2:] - ps[:-2]) / (ts[2:] - ts[:-2]) / ps[1:-1]
    late = (ts[1:-1] > 250.0)
    assert np.all(np.abs(p[late] + 3.0) < 0.1), p[late]


def test_quasinormal_ringing_in_rstar():
    """The r* system (BL time, field Phi = r Delta^s Psi) rings at the textbook
    fundamental quasinormal frequencies of tests/golden/qnm_frequencies.txt
    at r* = 50 M: Schwarzschild and Kerr a = 0.7, (l, m) = (2, 2), s = -2;
    Prony fit of order 6 of the sY_lm projection over t = 120..170 M (the
    boundaries at -100 M and 300 M are causally disconnected from it);
    |omega| within 0.5%, gamma within 1%."""
    from _qnm import golden_qnm, nearest_mode, prony_modes
    nr, nth, every = 1024, 16, 0.25
    h = 400.0 / (nr - 1)
    dth = np.pi / nth
    for s, l, m, a, wr, gam in golden_qnm():
        if s != -2 or a > 0.8:
            continue
        g = o.grid(nr, nth, -100.0, 300.0, 1.0, a, s, m, field=1)
        co = o.coefficients(g)
        kap = co[7] * 16 / 3 / dth ** 2 + np.abs(co[8]) * 1.5 / dth + np.hypot(co[5], co[6])
        dt = 0.5 / np.max(co[0] / h + np.sqrt(np.maximum(kap, 0.0)))
        n = int(np.ceil(every / dt))
        dt = every / n
        wl = I.KERR_GRAV.with_(nr=nr, nth=nth, a=a, s=s, m=m, ells=(l,), rc=30.0, width=3.0)
        u = I.initial_data(wl)
        th = I.theta_nodes(nth)
        w = I.swsh(s, l, m, th) * np.sin(th) * dth
        ie = int(round(150.0 / h))                       # r* = 50 M
        ts, ys, t = [], [], 0.0
        while t < 175.0:
            u = o.rk3_step(g, co, dt, u, n)
            t += n * dt
            ts.append(t)
            ys.append(np.sum(w * (u[0, :, ie] + 1j * u[1, :, ie])))
        gm, om = nearest_mode(prony_modes(np.array(ts), np.array(ys), 120.0, 170.0), wr, gam)
        assert abs(abs(om) - wr) < 5e-3 * wr, (a, om, wr)
        assert abs(gm - gam) < 1e-2 * gam, (a, gm, gam)
