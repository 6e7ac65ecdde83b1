"""Mistakes planted in the library's host coefficient generator, on the CPU:
each entry changes one thing in a copy of paper_2010_04760_gb300/csrc/
teuk_host.cpp (a flipped sign, a dropped or altered term, a wrong factor or
index), compiles the copy alone with the host C++ compiler, and compares the
coefficient planes it builds with the oracle's, as the host tests do. Every
planted mistake must be caught by that comparison and the unaltered copy must
pass it, so that the comparison ties each term of the product's generator (the
r* coefficients, the rescaled field, the hyperboloidal closed forms with their
hand-differentiated speed, the tortoise inversion and the theta stencil planes
with their pole parity) to the oracle, which its own pins tie to the paper.
The time-step rule is a reading, not a coefficient, and is not covered here."""
import concurrent.futures as cf
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as o
import paper_2010_04760_gb300 as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_04760_gb300", "csrc")
SRC = os.path.join(CSRC, "teuk_host.cpp")

# (name, text in teuk_host.cpp, replacement)
MUTANTS = [
    ("tortoise: sign of the extremal pole term", "- 2.0 * M * M / x;", "+ 2.0 * M * M / x;"),
    ("tortoise: sign of the r_- logarithm", "- km * std::log((x + w) / (2.0 * M));",
     "+ km * std::log((x + w) / (2.0 * M));"),
    ("b_*: sign of the Sigma^2 derivative", "(2.0 * r / varpi - 0.5 * dS2 * inv)",
     "(2.0 * r / varpi + 0.5 * dS2 * inv)"),
    ("dSigma^2/dr: sign of the a^2 term", "- 2.0 * a * a * (r - M) * sn * sn;",
     "+ 2.0 * a * a * (r - M) * sn * sn;"),
    ("B*: (r - M) written (r + M)",
     "const double Bs_r = (2.0 * r * Delta + 2.0 * s * (r - M) * varpi) * inv;",
     "const double Bs_r = (2.0 * r * Delta + 2.0 * s * (r + M) * varpi) * inv;"),
    ("Bt: sign of the s a Delta cos term", "-(4.0 * M * a * m * r + 2.0 * s * a * Delta * cs)",
     "-(4.0 * M * a * m * r - 2.0 * s * a * Delta * cs)"),
    ("C: sign of the pole potential", "c.Cr = Delta * (s - mc * mc / (sn * sn)) * inv;",
     "c.Cr = Delta * (s + mc * mc / (sn * sn)) * inv;"),
    ("C: (r - M) written r", "c.Ci = 4.0 * s * m * a * (r - M) * inv;",
     "c.Ci = 4.0 * s * m * a * r * inv;"),
    ("rescaled field: Delta/r written Delta in Im C", "c.Ci = -2.0 * m * a * Delta / r * inv;",
     "c.Ci = -2.0 * m * a * Delta * inv;"),
    ("rescaled field: (1 + s) M written s M", "- 2.0 * (1.0 + s) * M / r) * inv;",
     "- 2.0 * s * M / r) * inv;"),
    ("rescaled field: K built from Psi's B*", "c.Kr = Bsr - b * bstar - b * c.Btr;",
     "c.Kr = Bs_r - b * bstar - b * c.Btr;"),
    ("K: sign of b Im Bt", "c.Ki = Bs_i - b * c.Bti;", "c.Ki = Bs_i + b * c.Bti;"),
    ("hyperboloidal c: W for W^2", "c.c = W * W * E * invD;", "c.c = W * E * invD;"),
    ("hyperboloidal db/drho: sign of the E' term", "- c.b * E_r / E;", "+ c.b * E_r / E;"),
    ("hyperboloidal G': 4M/S for 2M/S", "rho * (1.0 + 2.0 * M / S +",
     "rho * (1.0 + 4.0 * M / S +"),
    ("hyperboloidal sigma': dropped factor 2", "(2.0 * x * x_r * delta + x * x * delta_r)",
     "(x * x_r * delta + x * x * delta_r)"),
    ("hyperboloidal B^rho: (1 + s) written (1 - s)", "(M * (1.0 + s) - a2 * x)",
     "(M * (1.0 - s) - a2 * x)"),
    ("hyperboloidal C: (s + 1) M written s M", "- 2.0 * (s + 1.0) * M * x",
     "- 2.0 * s * M * x"),
    ("hyperboloidal K: b for c in the last term", "c.Kr = Brr - c.b * c.Btr - c.c * b_r;",
     "c.Kr = Brr - c.b * c.Btr - c.b * b_r;"),
    ("hyperboloidal Bt: sign of (1 - H')", "c.Bti = (2.0 * m * a * (1.0 - Hp)",
     "c.Bti = (2.0 * m * a * (Hp - 1.0)"),
    ("theta planes: sign of B in the j-1 weight", "16.0 * A - 8.0 * B,", "16.0 * A + 8.0 * B,"),
    ("theta planes: pole parity inverted",
     "const double sigma = ((p->m + p->s) % 2 == 0) ? 1.0 : -1.0;",
     "const double sigma = ((p->m + p->s) % 2 == 0) ? -1.0 : 1.0;"),
    ("theta planes: pole mirror on the node", "if (jj < 0) tgt = -1 - jj;",
     "if (jj < 0) tgt = -jj;"),
    ("radial planes: dt/(3h) for dt/(6h)",
     "const double c6h = dt / ((p->scheme == TEUK_SCHEME_FD6_KO8 ? 60.0 : 6.0) * h);",
     "const double c6h = dt / ((p->scheme == TEUK_SCHEME_FD6_KO8 ? 60.0 : 3.0) * h);"),
    ("radial spacing over nr", "const double h = (p->rstar_max - p->rstar_min) / (nr - 1);",
     "const double h = (p->rstar_max - p->rstar_min) / nr;"),
]

R_CASES = [(0.999, -2, 2, 0), (0.4, -1, 1, 0), (1.0, 0, 0, 0), (0.7, 2, 3, 0),
           (0.999, -2, 2, 1), (0.7, 2, 3, 1)]            # (a, s, m, field)
HYP_CASES = [(1.0, -2, 0), (0.7, -2, 2), (0.3, 1, -1)]
NR, NTH, DT = 40, 12, 0.07


def _compile(tmp, tag, text):
    src = os.path.join(tmp, f"host_{tag}.cpp")
    with open(src, "w") as fh:
        fh.write(text)
    out = os.path.join(tmp, f"libhost_{tag}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", CSRC, src, "-o", out,
                           "-lpthread"])
    return out


def _builder(path):
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(T.teuk_params)
    L.teuk_coeff_count.argtypes, L.teuk_coeff_count.restype = [P], ctypes.c_size_t
    L.teuk_build_coefficients.argtypes = [P, ctypes.c_double, ctypes.c_void_p]
    L.teuk_build_coefficients.restype = ctypes.c_int

    def build(p, dt):
        n = L.teuk_coeff_count(ctypes.byref(p))
        out = np.zeros((n // (p.nr * p.ntheta), p.ntheta, p.nr))
        st = L.teuk_build_coefficients(ctypes.byref(p), dt, out.ctypes.data_as(ctypes.c_void_p))
        if st != 0 or not np.all(np.isfinite(out)):
            return None
        return out
    return build


def _close(got, ref, rtol, atol):
    return got.shape == ref.shape and bool(np.all(np.abs(got - ref) <= atol + rtol * np.abs(ref)))


def _theta_planes_ok(got, co, s, m, dt):
    """The five theta planes, applied to a field with the pole parity, must
    give dt (Ath Psi_thth + Bth Psi_th + Re C Psi) of the oracle's centred
    ghost-row operator."""
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth = co[:9]
    dth = np.pi / NTH
    psi = np.random.default_rng(0).standard_normal((NTH, NR))
    sig = 1.0 if (m + s) % 2 == 0 else -1.0
    acc = np.zeros((NTH, NR))
    for k in range(-2, 3):
        rows = np.clip(np.arange(NTH) + k, 0, NTH - 1)
        acc += got[8 + k] * psi[rows]
    ext = np.concatenate([sig * psi[1::-1], psi, sig * psi[:-3:-1]])
    nb = [ext[2 + k:2 + k + NTH] for k in range(-2, 3)]
    th1 = (nb[0] - 8 * nb[1] + 8 * nb[3] - nb[4]) / (12 * dth)
    th2 = (-nb[0] + 16 * nb[1] - 30 * nb[2] + 16 * nb[3] - nb[4]) / (12 * dth ** 2)
    exp_ = DT * (Ath * th2 + Bth * th1 + Cr * psi)
    return _close(acc, exp_, 1e-8, 1e-10 * np.max(np.abs(exp_)))


def _mismatches(build, refs):
    """Names of the cases whose planes differ from the oracle's."""
    bad = []
    for name, p, co, coords, s, m in refs:
        got = build(p, DT)
        if got is None:
            bad.append(name + ": failed")
            continue
        b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth, c = co
        h = (p.rstar_max - p.rstar_min) / (p.nr - 1)
        atol = 1e-13 * DT * np.max(np.abs(co)) / h
        pairs = [(0, DT * b / (6 * h)), (1, DT * Kr / (6 * h)), (2, DT * Ki / (6 * h)),
                 (3, DT * Br), (4, DT * Bi), (5, DT * Ci)]
        if coords == 1:
            pairs.append((12, DT * c / (6 * h)))
        if not all(_close(got[k], ref, 1e-9, atol) for k, ref in pairs):
            bad.append(name + ": radial planes")
        elif not _theta_planes_ok(got, co, s, m, DT):
            bad.append(name + ": theta planes")
    return bad


def _references():
    refs = []
    for a, s, m, field in R_CASES:
        p = T.make_params(NR, NTH, -60.0, 120.0, 1.0, a, s, m, field=field)
        co = o.coefficients(o.grid(NR, NTH, -60.0, 120.0, 1.0, a, s, m, field=field))
        refs.append((f"r* a={a} s={s} m={m} field={field}", p, co, 0, s, m))
    for a, s, m in HYP_CASES:
        p = T.make_params(NR, NTH, a=a, s=s, m=m, coords=T.TEUK_COORDS_HYPERBOLOIDAL, hyp_S=20.0)
        g = o.grid(NR, NTH, p.rstar_min, p.rstar_max, 1.0, a, s, m, coords=1, S=20.0)
        refs.append((f"hyperboloidal a={a} s={s} m={m}", p, o.coefficients(g), 1, s, m))
    return refs


def test_host_mutants_are_distinct_single_edits():
    text = open(SRC).read()
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)
    for name, old, new in MUTANTS:
        assert text.count(old) == 1, name
        assert old != new, name


@pytest.mark.slow
def test_every_planted_host_mistake_is_caught_by_the_oracle_comparison(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    text = open(SRC).read()
    tmp = str(tmp_path)
    texts = [text] + [text.replace(old, new) for _, old, new in MUTANTS]
    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        libs = list(ex.map(lambda a: _compile(tmp, *a),
                           [(str(k), t) for k, t in enumerate(texts)]))
    refs = _references()
    assert _mismatches(_builder(libs[0]), refs) == [], "the unaltered generator disagrees"
    survivors = [name for (name, _, _), lib in zip(MUTANTS, libs[1:])
                 if not _mismatches(_builder(lib), refs)]
    assert not survivors, survivors
