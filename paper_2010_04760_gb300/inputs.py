"""Seeded synthetic inputs for the WENO5 Teukolsky evolutions.

This module holds only grid nodes and initial data; none of the solver's
arithmetic lives here. Both the CUDA path's tests/benchmarks and the oracle
checks draw their inputs from it, so the two sides see identical data.

Initial data (the paper's own run uses a Gaussian wave packet times a
spherical harmonic, Sec. 4): Psi(x, theta) = sum_l A_l exp(i phi_l)
exp(-(x - rc)^2 / (2 w^2)) sY_lm(theta), pi = 0, with x the radial coordinate
(r*, or rho on the hyperboloidal slices, where Psi stands for the evolved
Phi = r Delta^s Psi). Amplitudes A_l ~ U(0.5, 1.5) and phases
phi_l ~ U(0, 2 pi) come from ``numpy.random.default_rng(seed)``. The width w
is the Gaussian's standard deviation.

Grid: x_i = rs_min + i h, h = (rs_max - rs_min)/(nr - 1), i = 0..nr-1;
theta_j = (j + 1/2) pi / nth (cell centred).
"""
from dataclasses import dataclass, field, replace
from math import comb, factorial, pi, sqrt

import numpy as np

DEFAULT_RSTAR = (-100.0, 300.0)


def rstar_nodes(nr, rs_min, rs_max):
    return rs_min + np.arange(nr) * ((rs_max - rs_min) / (nr - 1))


def theta_nodes(nth):
    return (np.arange(nth) + 0.5) * (pi / nth)


def swsh(s, l, m, theta):
    """Spin-weighted spherical harmonic sY_lm(theta, phi=0) (Goldberg et al.
    1967 sum formula). sin^(2l)(x) cot^k(x) is evaluated as sin^(2l-k) cos^k
    with x = theta/2; every power that occurs is non-negative."""
    if l < max(abs(s), abs(m)):
        raise ValueError("need l >= max(|s|, |m|)")
    x = 0.5 * np.asarray(theta, dtype=np.float64)
    sx, cx = np.sin(x), np.cos(x)
    norm = sqrt(factorial(l + m) * factorial(l - m) * (2 * l + 1)
                / (4 * pi * factorial(l + s) * factorial(l - s)))
    total = np.zeros_like(x)
    for r in range(0, l - s + 1):
        k2 = r + s - m
        if k2 < 0 or k2 > l + s:
            continue
        k = 2 * r + s - m
        term = comb(l - s, r) * comb(l + s, k2) * (-1.0) ** (l - r - s)
        total = total + term * sx ** (2 * l - k) * cx ** k
    return (-1.0) ** m * norm * total


@dataclass(frozen=True)
class Workload:
    """One evolution: grid, black hole, mode, weights and initial data."""
    name: str
    nr: int
    nth: int
    rs_min: float = DEFAULT_RSTAR[0]
    rs_max: float = DEFAULT_RSTAR[1]
    M: float = 1.0
    a: float = 0.0
    s: int = 0
    m: int = 0
    wprec: str = "fp64"
    cfl: float = 0.5
    eps: float = 1e-6
    rc: float = 50.0
    width: float = 4.0
    ells: tuple = (2,)
    seed: int = 0
    t_end: float = 0.0
    nsteps: int = 0
    extra: dict = field(default_factory=dict)
    coords: int = 0          # 0: BL t and r*; 1: hyperboloidal (tau, rho)
    field: int = None        # evolved field (None: Psi in r*, Phi on the slices)
    S: float = 20.0          # hyperboloidal slice parameter

    def with_(self, **kw):
        return replace(self, **kw)

    @property
    def points(self):
        return self.nr * self.nth


def initial_data(w: Workload):
    """u[4, nth, nr] = (Re Psi, Im Psi, Re pi, Im pi) with pi = 0."""
    rng = np.random.default_rng(w.seed)
    rs = rstar_nodes(w.nr, w.rs_min, w.rs_max)
    th = theta_nodes(w.nth)
    radial = np.exp(-0.5 * ((rs - w.rc) / w.width) ** 2)
    psi = np.zeros((w.nth, w.nr), dtype=np.complex128)
    for l in w.ells:
        amp = rng.uniform(0.5, 1.5)
        phase = rng.uniform(0.0, 2 * pi)
        ang = swsh(w.s, l, w.m, th)
        psi += amp * np.exp(1j * phase) * np.outer(ang, radial)
    u = np.zeros((4, w.nth, w.nr))
    u[0], u[1] = psi.real, psi.imag
    return u


def splitmix64_uniforms(seed, count):
    """Uniforms in [0, 1) from SplitMix64 (Steele, Lea, Flood 2014):
    u = (x >> 11) 2^-53 for each 64-bit output x."""
    mask = (1 << 64) - 1
    state = seed & mask
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z = z ^ (z >> 31)
        out.append((z >> 11) * 2.0 ** -53)
    return out


def gaussian_data(w: Workload, rc, width, coeffs):
    """u[4, nth, nr]: Psi = sum_k coeffs[k] exp(-(r* - rc)^2 / (2 width^2))
    sY_{l0+k, m}(theta) with l0 = max(|s|, |m|), pi = 0."""
    rs = rstar_nodes(w.nr, w.rs_min, w.rs_max)
    th = theta_nodes(w.nth)
    radial = np.exp(-0.5 * ((rs - rc) / width) ** 2)
    l0 = max(abs(w.s), abs(w.m))
    ang = sum(c * swsh(w.s, l0 + k, w.m, th) for k, c in enumerate(coeffs))
    psi = np.outer(ang, radial)
    u = np.zeros((4, w.nth, w.nr))
    u[0], u[1] = psi.real, psi.imag
    return u


def random_state(nr, nth, seed, smooth=True):
    """A generic seeded state for operator-level parity checks: a sum of a
    few Gaussians and sinusoids in r* times smooth theta profiles, plus (if
    smooth is False) jumps that switch the nonlinear weights."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, nr)
    th = theta_nodes(nth)
    u = np.zeros((4, nth, nr))
    for c in range(4):
        for _ in range(3):
            amp = rng.uniform(-1.0, 1.0)
            xc = rng.uniform(0.1, 0.9)
            wd = rng.uniform(0.02, 0.2)
            kt = rng.integers(0, 4)
            u[c] += amp * np.outer(np.cos(kt * th + rng.uniform(0, pi)),
                                   np.exp(-0.5 * ((x - xc) / wd) ** 2))
        u[c] += 0.1 * rng.uniform(-1, 1) * np.outer(np.sin(th), np.sin(7 * pi * x))
        if not smooth:
            for _ in range(2):
                xj = rng.uniform(0.1, 0.9)
                u[c] += rng.uniform(-1, 1) * (x[None, :] > xj) * np.cos(th)[:, None]
    return u


def multiscale_state(nr, nth, seed, smooth=True):
    """random_state with every theta row scaled by 10^U(-40, 6) and the first
    nr/8 radial nodes by a further 1e-200: regions where epsilon dominates the
    smoothness indicators and where the reduced-precision weights need their
    scaling into range."""
    u = random_state(nr, nth, seed, smooth=smooth)
    rng = np.random.default_rng(seed + 100)
    u = u * 10.0 ** rng.uniform(-40, 6, size=(1, nth, 1))
    u[:, :, : nr // 8] *= 1e-200
    return u


# ---------------------------------------------------------------------------
# Named workloads (sizes, physics and data of the benchmark suite).
# ---------------------------------------------------------------------------
SCHW_SCALAR = Workload(
    name="schwarzschild_s0_m0_256x32", nr=256, nth=32, a=0.0, s=0, m=0,
    wprec="fp64", cfl=0.5, rc=50.0, width=4.0, ells=(2,), seed=0, nsteps=500)

KERR_GRAV = Workload(
    name="kerr_a0.999_s-2_m2_2048x128", nr=2048, nth=128, a=0.999, s=-2, m=2,
    wprec="fp32", cfl=0.5, rc=30.0, width=3.0, ells=(2,), seed=1, t_end=500.0)

EXTREMAL_SCALAR = Workload(
    name="extremal_s0_m0_8192x256", nr=8192, nth=256, a=1.0, s=0, m=0,
    wprec="fp16", cfl=0.5, rc=-20.0, width=4.0, ells=(0, 2), seed=2, t_end=2000.0)

TAIL_SCALAR = Workload(
    name="tail_s0_m0_16384x512", nr=16384, nth=512, rs_min=-5000.0, rs_max=5000.0,
    a=0.0, s=0, m=0, wprec="fp32", cfl=0.5, rc=50.0, width=4.0, ells=(0,), seed=3,
    t_end=1.0e4)


def horizon_rho(M, a, S):
    """rho of the outer horizon r_+ = M + sqrt(M^2 - a^2) on the slices."""
    rp = M + sqrt(max(M * M - a * a, 0.0))
    return rp * S / (rp + S)


# The paper's own run (Sec. 4): extremal Kerr (a = M), s = -2, (l, m) = (2, 0),
# a wave packet at rho = 1.0 of width 0.22 on the hyperboloidal slices with
# S = 20, 16384 (rho) x 64 (theta) nodes from the horizon to scri.
EXTREMAL_GRAV_HYP = Workload(
    name="extremal_hyp_s-2_m0_16384x64", nr=16384, nth=64,
    rs_min=horizon_rho(1.0, 1.0, 20.0), rs_max=20.0, a=1.0, s=-2, m=0,
    wprec="fp32", cfl=0.5, rc=1.0, width=0.22, ells=(2,), seed=4, t_end=1000.0,
    coords=1, S=20.0)


def batch_workloads(n=64, seed=2026):
    """Uneven batch: nr uniform over multiples of 128 in [1024, 8192], nth over
    multiples of 16 in [64, 256], a ~ U[0, M], s in {0, -2}, m in {0..4}."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nr = int(rng.integers(8, 65)) * 128
        nth = int(rng.integers(4, 17)) * 16
        a = float(rng.uniform(0.0, 1.0))
        s = int(rng.choice([0, -2]))
        m = int(rng.integers(0, 5))
        l = max(2, abs(m), abs(s))
        out.append(Workload(name=f"batch{k}", nr=nr, nth=nth, a=a, s=s, m=m,
                            wprec="fp32", rc=30.0, width=3.0, ells=(l,),
                            seed=seed + k))
    return out
