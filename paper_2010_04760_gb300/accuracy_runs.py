"""Long evolutions of the two large workloads, comparing weight formats.

    python -m paper_2010_04760_gb300.accuracy_runs extremal --wprec fp16 \\
        --t-end 2000 --out extremal_fp16.npz
    python -m paper_2010_04760_gb300.accuracy_runs tail --wprec fp32 --a 0 \\
        --t-end 1000 --out tail_fp32.npz
    python -m paper_2010_04760_gb300.accuracy_runs compare A.npz B.npz

extremal: the extremal scalar (a = M, s = m = 0) on 8192 (r* in [-100, 300] M)
x 256 (theta) nodes, l = 0 + 2 packet at r* = -20 M, at the stability rule's
time step. Every `--every` steps the horizon gather (Psi, pi and dPsi/dr* at
the innermost node, every theta row; Sec. 4's observables read in r*, where
the horizon itself is at r* = -infinity) is recorded, with the l = 0
projection of dPsi/dr* there, sum_j dPsi/dr*(theta_j) sin(theta_j) dtheta / 2,
as the horizon charge proxy H(t).

tail: the tail workload (s = m = 0, l = 0 pulse at r* = 50 M, r* in [-5000,
5000] M) on 16384 x 512 nodes, time step 10/n (n steps per 10 M, from the
stability rule), Psi at r* = 50 M recorded every 10 M (theta row nth/2).

Each run writes an .npz with the time series and the run's parameters (the
file is rewritten every `--save-every` samples, so a run cut short keeps what
it did). `compare` prints the relative L2 difference of the recorded series
of two runs and, for the tail, the local index p = t dPsi/dt / Psi of each
(central differences over +-10 M) every 100 M.
"""
import argparse
import json
import sys
import time

import numpy as np

from . import inputs as I
from . import params_from_workload, teuk_create, teuk_get_info, teuk_observe, teuk_set_state
from . import teuk_stable_dt, teuk_step


def _save(path, **arrays):
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    import os
    os.replace(tmp, path)


def run_extremal(wprec, t_end, every, out, save_every=20):
    wl = I.EXTREMAL_SCALAR
    p = params_from_workload(wl, wprec=wprec)
    h = teuk_create(p)
    teuk_set_state(h, I.initial_data(wl), 0.0)
    _, dt, _ = teuk_get_info(h)
    th = I.theta_nodes(wl.nth)
    wq = np.sin(th) * (np.pi / wl.nth) / 2.0           # l = 0 projection weights
    nsamp = int(t_end / (dt * every))
    ts, hor, charge = [], [], []
    t0 = time.perf_counter()
    for k in range(nsamp):
        teuk_step(h, every)
        _, hz, t = teuk_observe(h, 0.0)
        ts.append(t)
        hor.append(hz.copy())
        charge.append(np.sum(wq * hz[:, 4]))
        if (k + 1) % save_every == 0 or k + 1 == nsamp:
            _save(out, t=np.array(ts), horizon=np.array(hor), charge=np.array(charge),
                  meta=json.dumps({"workload": wl.name, "wprec": wprec, "dt": dt,
                                   "every": every, "t_end": t_end,
                                   "seconds": time.perf_counter() - t0}))
    h.close()
    return out


def run_tail(wprec, a, t_end, out, save_every=10):
    wl = I.TAIL_SCALAR.with_(a=float(a))
    dt_rule = teuk_stable_dt(params_from_workload(wl, wprec=wprec))
    n = int(np.ceil(10.0 / dt_rule))                   # steps per 10 M
    dt = 10.0 / n
    p = params_from_workload(wl, wprec=wprec, dt=dt)
    h = teuk_create(p)
    teuk_set_state(h, I.initial_data(wl), 0.0)
    nsamp = int(round(t_end / 10.0))
    ts, psi = [], []
    t0 = time.perf_counter()
    for k in range(nsamp):
        teuk_step(h, n)
        wave, _, t = teuk_observe(h, 50.0)
        ts.append(t)
        psi.append(wave[wl.nth // 2].copy())
        if (k + 1) % save_every == 0 or k + 1 == nsamp:
            _save(out, t=np.array(ts), psi=np.array(psi),
                  meta=json.dumps({"workload": wl.name, "a": a, "wprec": wprec, "dt": dt,
                                   "steps_per_10M": n, "t_end": t_end,
                                   "seconds": time.perf_counter() - t0}))
    h.close()
    return out


def local_index(t, y, stride=1):
    """p = t dy/dt / y by central differences over +-stride samples."""
    p = np.full(len(t), np.nan)
    for k in range(stride, len(t) - stride):
        p[k] = t[k] * (y[k + stride] - y[k - stride]) / ((t[k + stride] - t[k - stride]) * y[k])
    return p


def compare(a_path, b_path):
    A, B = np.load(a_path), np.load(b_path)
    ma, mb = json.loads(str(A["meta"])), json.loads(str(B["meta"]))
    n = min(len(A["t"]), len(B["t"]))
    res = {"a": ma, "b": mb, "samples": n, "t_last": float(A["t"][n - 1])}
    if "horizon" in A:
        ha, hb = A["horizon"][:n], B["horizon"][:n]
        res["horizon_rel_l2"] = float(np.linalg.norm(ha - hb) / np.linalg.norm(hb))
        ca, cb = A["charge"][:n], B["charge"][:n]
        res["charge_max_rel_diff"] = float(np.max(np.abs(ca - cb)) / np.max(np.abs(cb)))
        res["charge_b_first_last"] = [float(cb[0]), float(cb[-1])]
    else:
        ya, yb = A["psi"][:n, 0], B["psi"][:n, 0]
        res["psi_rel_l2"] = float(np.linalg.norm(ya - yb) / np.linalg.norm(yb))
        t = A["t"][:n]
        pa, pb = local_index(t, ya), local_index(t, yb)
        pick = [k for k in range(n) if abs(t[k] % 100.0) < 1e-6 or abs(t[k] % 100.0 - 100) < 1e-6]
        res["index_every_100M"] = [[float(t[k]), float(pa[k]), float(pb[k])] for k in pick]
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["extremal", "tail", "compare"])
    ap.add_argument("files", nargs="*")
    ap.add_argument("--wprec", default="fp32")
    ap.add_argument("--a", type=float, default=0.0)
    ap.add_argument("--t-end", type=float, default=100.0)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    if args.what == "compare":
        print(json.dumps(compare(*args.files), indent=1))
        return
    import torch
    torch.cuda.set_device(0)
    out = args.out or f"{args.what}_{args.wprec}.npz"
    t0 = time.perf_counter()
    if args.what == "extremal":
        run_extremal(args.wprec, args.t_end, args.every, out)
    else:
        run_tail(args.wprec, args.a, args.t_end, out)
    print(f"{args.what} {args.wprec} a={args.a} t_end={args.t_end}: "
          f"{time.perf_counter() - t0:.1f} s -> {out}", flush=True)


if __name__ == "__main__":
    sys.exit(main())
