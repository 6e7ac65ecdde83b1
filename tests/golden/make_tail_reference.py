"""Writes tests/golden/tail_coarse_reference.txt: the CPU oracle's late-time
tail of the 16384 x 512 tail workload (s = m = 0, l = 0 pulse at r* = 50 M,
r* in [-5000, 5000] M) on a coarsened grid, 4096 (r*, 4x coarser) x 8 (theta:
the l = 0 data needs few rows, and 128 rows would force a time step 40x
smaller through the theta part near the hole), evolved with binary64 weights
and SSP-RK(3,3) to t = 10^4 M, for a = 0 and a = M. The time step is the
stability rule (cfl 0.5) evaluated on the oracle's coefficients, rounded down
to 100/n. Recorded every 100 M: t, Psi at r* = 50 M (theta row 4) and the local
index p = t dPsi/dt / Psi (central differences). Price's law gives p -> -3 at
a = 0 (and away from the horizon at a = M). The pulse's reflection from the
outer end (r* = 5000 M) returns to r* = 50 M at t ~ 9900 M, so the tail is read
before that.

With --ld the state, weights and fluxes are carried in C long double by the
extended-precision oracle instead (same grid, coefficients, time step and
initial data), written to tail_coarse_reference_ld.txt: the difference of the
two files is the binary64 state's own round-off along the tail.

Calls only the oracle and the seeded inputs:
    python tests/golden/make_tail_reference.py        # about 10 min on 8 cores
    python tests/golden/make_tail_reference.py --ld   # about 20 min on 8 cores
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as o                                      # noqa: E402
from paper_2010_04760_gb300 import inputs as I          # noqa: E402

NR, NTH, T_END, EVERY = 4096, 8, 1.0e4, 100.0
R_EXT = 50.0


def coarse_workload(a):
    return I.TAIL_SCALAR.with_(nr=NR, nth=NTH, a=a)


def time_step(g, co):
    """cfl 0.5 over max(|b|, |c|)/h + sqrt(theta frequencies), then EVERY/n."""
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth, c = co
    h = (g.rs_max - g.rs_min) / (g.nr - 1)
    dth = np.pi / g.nth
    kap = Ath * (16 / 3) / dth ** 2 + np.abs(Bth) * 1.5 / dth + np.hypot(Cr, Ci)
    dt = 0.5 / np.max(np.maximum(np.abs(b), np.abs(c)) / h + np.sqrt(np.maximum(kap, 0.0)))
    n = int(np.ceil(EVERY / dt))
    return EVERY / n, n


def run(a, ld=False):
    wl = coarse_workload(a)
    g = o.grid(NR, NTH, wl.rs_min, wl.rs_max, 1.0, a, 0, 0)
    co = o.coefficients(g)
    u = I.initial_data(wl)
    if ld:
        u = u.astype(np.longdouble)
    step = o.ld_rk3_step if ld else o.rk3_step
    h = (wl.rs_max - wl.rs_min) / (NR - 1)
    ie = int(round((R_EXT - wl.rs_min) / h))
    DT, n = time_step(g, co)
    print(f"a={a} dt={DT}", flush=True)
    ts, ys = [], []
    t = 0.0
    while t < T_END - 1e-9:
        u = step(g, co, DT, u, n)
        t += n * DT
        ts.append(t)
        ys.append(u[0, NTH // 2, ie])
        print(f"a={a} t={t:.0f}", flush=True)
    ts, ys = np.array(ts), np.array(ys, dtype=u.dtype)
    p = np.full_like(ts, np.nan)
    p[1:-1] = ts[1:-1] * (ys[2:] - ys[:-2]) / (ts[2:] - ts[:-2]) / ys[1:-1]
    return ts, ys, p


def main():
    ld = "--ld" in sys.argv[1:]
    rows = []
    for a in (0.0, 1.0):
        ts, ys, p = run(a, ld)
        rows += [(a, t, y, q) for t, y, q in zip(ts, ys, p)]
    out = os.path.join(HERE, "tail_coarse_reference_ld.txt" if ld else "tail_coarse_reference.txt")
    with open(out, "w") as fh:
        if ld:
            fh.write("# Extended-precision oracle reference (state, weights and fluxes in C long\n"
                     f"# double, {o.ld_mant_dig()}-bit significand; SSP-RK(3,3), stability-rule dt)\n"
                     "# for the tail workload coarsened to 4096 x 8 (r* in [-5000, 5000] M,\n"
                     "# s = m = 0, l = 0 pulse at 50 M): Psi at r* = 50 M, theta row 4, every\n"
                     "# 100 M, and the local index p = t dPsi/dt / Psi. Written by\n"
                     "# tests/golden/make_tail_reference.py --ld (oracle and seeded inputs only).\n"
                     "# columns: a  t  Psi  p\n")
            for a, t, y, q in rows:
                fh.write(f"{a:.1f} {t:.1f} "
                         f"{np.format_float_scientific(y, precision=20, unique=False)} "
                         f"{float(q):.10f}\n")
        else:
            fh.write("# Oracle reference (binary64 weights, SSP-RK(3,3), stability-rule dt) for\n"
                     "# the tail workload coarsened to 4096 x 8 (r* in [-5000, 5000] M, s = m = 0,\n"
                     "# l = 0 pulse at 50 M): Psi at r* = 50 M, theta row 4, every 100 M, and the\n"
                     "# local index p = t dPsi/dt / Psi. Written by\n"
                     "# tests/golden/make_tail_reference.py (oracle and seeded inputs only).\n"
                     "# columns: a  t  Psi  p\n")
            for a, t, y, q in rows:
                fh.write(f"{a:.1f} {t:.1f} {y:.17e} {q:.10f}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
