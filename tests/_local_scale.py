"""Per-node tolerance scale for comparing the CUDA path with the oracle.

Round-off of a correctly implemented stage is relative to the size of the
terms that enter each output node, not to the largest value anywhere on the
grid. This module bounds those terms node by node from the oracle's own
coefficient planes (b, K, Bt, C, Ath, Bth, c) and the input state, so that
low-amplitude regions (rows scaled down by 1e-40, a 1e-200 tail, the far
field of a pulse) are checked at their own scale:

  radial part (WENO5 or FD6): R / h times the speed (b, c) or the coupling
    (|K|), with R the largest |u| of the component over the node's radial
    stencil (+-3 nodes, +-4 for FD6 + KO8); the Kreiss-Oliger term adds
    sigma R / h;
  theta part: (|Ath| 64/(12 dth^2) + |Bth| 18/(12 dth)) times the largest |Psi|
    over the rows j-2..j+2 (the absolute weights of the fourth-order centred
    stencils), plus |Bth| Theta/dth for the theta-WENO option (rows j-3..j+3);
  zeroth-order couplings: |Bt| |pi|, |C| |Psi|, and |pi| in the Psi rows.

The intermediates of the flux form reach 72 R in units of 6h (|D| <= 12 R/h),
so binary64 round-off of a stage stays below ~1e-14 of this scale.

On the hyperboloidal slices the radial ghosts extrapolate the quartic through
the five edge nodes; a ghost n nodes out is bounded by the Lebesgue sum
sum_k |l_k(-n)| of that extrapolation times the largest edge value, which
enters R near either end.

Each coefficient is itself known only to the round-off of the terms it is
made of: a coefficient that vanishes somewhere through cancellation (b on the
horizon, K next to it, where B*, b b_* and b Bt cancel) carries an absolute
error of about 2^-52 times the size of those terms whichever way it is
evaluated. So besides the scale S (compared at 1e-12) every term contributes
with its coefficient replaced by that coefficient's largest size on the grid
to a second scale S_c, compared at COEF_EPS = 2^-52: the bound at a node is
1e-12 S + COEF_EPS S_c (+ 1e-300).

A stage u_out = alpha u^n + beta (u_prev + dt F(u_prev)) has the scale
alpha |u^n| + beta (|u_prev| + dt S_F). For several steps the one-stage scale
of the initial state is spread over the domain of dependence of the run (the
radial and theta stencil reach times the number of stages).
"""
import numpy as np


def _lebesgue_ghost(n):
    """sum_k |l_k(-n)|, l_k the Lagrange basis of the nodes 0..4."""
    x = -float(n)
    tot = 0.0
    for k in range(5):
        lk = 1.0
        for m in range(5):
            if m != k:
                lk *= (x - m) / (k - m)
        tot += abs(lk)
    return tot


def _radial_env(a, halo, hyp):
    """max |a| over i-halo..i+halo along the last axis, ghosts included."""
    a = np.abs(a)
    nr = a.shape[-1]
    if hyp:
        left = np.max(a[..., :5], axis=-1, keepdims=True)
        right = np.max(a[..., nr - 5:], axis=-1, keepdims=True)
        gl = [left * _lebesgue_ghost(n) for n in range(halo, 0, -1)]
        gr = [right * _lebesgue_ghost(n) for n in range(1, halo + 1)]
    else:
        gl = [a[..., :1]] * halo
        gr = [a[..., nr - 1:]] * halo
    p = np.concatenate(gl + [a] + gr, axis=-1)
    out = p[..., 0:nr].copy()
    for s in range(1, 2 * halo + 1):
        np.maximum(out, p[..., s:s + nr], out=out)
    return out


def _theta_env(a, reach):
    """max |a| over rows j-reach..j+reach (clamped: rows mirrored across a pole
    are rows 0..reach-1 or their far-pole counterparts, all inside the clamp)."""
    a = np.abs(a)
    nth = a.shape[-2]
    if reach >= nth - 1:
        return np.broadcast_to(np.max(a, axis=-2, keepdims=True), a.shape).copy()
    out = a.copy()
    for k in range(1, reach + 1):
        lo = np.concatenate([a[..., :1, :]] * k + [a[..., :nth - k, :]], axis=-2)
        hi = np.concatenate([a[..., k:, :]] + [a[..., nth - 1:, :]] * k, axis=-2)
        np.maximum(out, lo, out=out)
        np.maximum(out, hi, out=out)
    return out


def _spread(a, rad, th):
    """max of a over the box i-rad..i+rad, j-th..j+th (clamped)."""
    out = _radial_env(a, rad, hyp=False) if rad > 0 else np.abs(a)
    return _theta_env(out, th) if th > 0 else out


def _terms(g, co, u):
    """The terms entering F(u) at every node, as (coefficient, operand) pairs
    per output component: coefficient magnitudes [nth, nr] and operand sizes."""
    hyp = int(g.coords) == 1
    fd6 = int(g.scheme) == 1
    h = (g.rs_max - g.rs_min) / (g.nr - 1)
    dth = np.pi / g.nth
    halo = 4 if fd6 else 3
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth = (np.abs(x) for x in co[:9])
    c = np.abs(co[9]) if co.shape[0] > 9 else b
    K, Bt, C = Kr + Ki, Br + Bi, Cr + Ci
    R = _radial_env(u, halo, hyp)
    D = R / h
    au = np.abs(u)
    one = np.ones_like(b)
    th2, th1 = (64.0 / 12.0) / dth ** 2, (18.0 / 12.0) / dth
    T0, T1 = _theta_env(u[0], 2), _theta_env(u[1], 2)
    psi_rows = [[(one, au[2]), (b, D[0])], [(one, au[3]), (b, D[1])]]
    common = [(K, D[0] + D[1]), (Bt, au[2] + au[3]), (C, au[0] + au[1])]
    pi_rows = [[(c, D[2])] + common + [(Ath, th2 * T0), (Bth, th1 * T0)],
               [(c, D[3])] + common + [(Ath, th2 * T1), (Bth, th1 * T1)]]
    if int(g.theta_mode) == 1:
        pi_rows[0].append((Bth, _theta_env(u[0], 3) / dth))
        pi_rows[1].append((Bth, _theta_env(u[1], 3) / dth))
    rows = psi_rows + pi_rows
    if fd6:
        for r, k in zip(rows, range(4)):
            r.append((float(g.ko_sigma) * one, R[k] / h))
    return rows


def rhs_scale(g, co, u):
    """(S, S_c)[4, nth, nr]: the size of the terms entering F(u) at every node,
    with each coefficient's own size (S) and with its largest size on the
    grid (S_c, for the coefficient's round-off)."""
    S = np.zeros_like(u)
    Sc = np.zeros_like(u)
    for k, row in enumerate(_terms(g, co, u)):
        for coef, op in row:
            S[k] += coef * op
            Sc[k] += np.max(coef) * op
    return S, Sc


def stage_scale(g, co, dt, u_prev, u_n=None, alpha=0.0, beta=1.0, with_prev=True):
    """Scale pair of alpha u_n + beta (u_prev + dt F(u_prev)) (with_prev=False:
    the operator alone, dt F)."""
    S, Sc = rhs_scale(g, co, u_prev)
    S, Sc = beta * dt * S, beta * dt * Sc
    if with_prev:
        S = S + beta * np.abs(u_prev)
    if u_n is not None and alpha != 0.0:
        S = S + alpha * np.abs(u_n)
    return S, Sc


def run_scale(g, co, dt, u0, stages):
    """Scale pair of a state after `stages` Runge-Kutta stages from u0: the
    one-stage scales of u0 spread over the run's domain of dependence."""
    rad = (4 if int(g.scheme) == 1 else 3) * stages
    th = (3 if int(g.theta_mode) == 1 else 2) * stages
    out = []
    for part in stage_scale(g, co, dt, u0):
        spread = _spread(np.maximum.reduce(part, axis=0)[None], rad, th)[0]
        out.append(np.broadcast_to(spread, part.shape).copy())
    return tuple(out)


FLOOR = 1e-300      # absolute floor: the bottom of binary64's normal range
COEF_EPS = 2.0 ** -52


def assert_local(got, exp_, scale, tol=1e-12, what=""):
    """|got - exp| <= tol * S + COEF_EPS * S_c + FLOOR at every node and
    component (scale = (S, S_c)); on failure, report the worst node."""
    S, Sc = scale
    err = np.abs(got - exp_)
    bound = tol * S + COEF_EPS * Sc + FLOOR
    bad = err > bound
    if np.any(bad):
        ratio = np.where(bad, err / bound, 0.0)
        c, j, i = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
        raise AssertionError(
            f"{what}: {int(bad.sum())} nodes over the local bound; worst component {c} "
            f"row {j} node {i}: got {got[c, j, i]!r} expected {exp_[c, j, i]!r} "
            f"err {err[c, j, i]:.3e} bound {bound[c, j, i]:.3e} (S {S[c, j, i]:.3e}, "
            f"S_c {Sc[c, j, i]:.3e})")
