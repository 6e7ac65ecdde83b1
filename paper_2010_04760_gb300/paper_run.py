"""The paper's own evolution (Sec. 4): extremal Kerr (a = M), s = -2,
(l, m) = (2, 0), a wave packet at rho = 1 on the hyperboloidal slices of
Sec. 2.2 (S = 20 M, horizon to scri), binary32 weights by default.

    python -m paper_2010_04760_gb300.paper_run --tau 200 --every 10

prints, every `every` M of tau, Phi and dPhi/drho on the horizon (the
Aretakis observables of Sec. 4, middle theta row), Phi at scri and the local
decay index tau dPhi/dtau / Phi on the horizon, then the throughput of the
stepping in point-stage updates per second. Runs on cuda:0 through the C ABI.
`--scheme fd6` runs the paper's comparison scheme instead (sixth-order centred
differences with Kreiss-Oliger dissipation of strength `--sigma`, Sec. 3.1.1).
"""
import argparse
import time

import numpy as np

from . import inputs as I
from . import teuk_create, teuk_get_info, teuk_observe, teuk_set_state, teuk_step
from . import TEUK_SCHEME_FD6_KO8, TEUK_SCHEME_WENO5, params_from_workload


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--nr", type=int, default=I.EXTREMAL_GRAV_HYP.nr)
    ap.add_argument("--nth", type=int, default=I.EXTREMAL_GRAV_HYP.nth)
    ap.add_argument("--wprec", default=I.EXTREMAL_GRAV_HYP.wprec,
                    choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--tau", type=float, default=50.0, help="final tau (units of M)")
    ap.add_argument("--steps", type=int, default=0, help="run this many steps instead")
    ap.add_argument("--every", type=float, default=10.0, help="observation interval in tau")
    ap.add_argument("--scheme", default="weno5", choices=["weno5", "fd6"],
                    help="radial scheme: WENO5 or FD6 + Kreiss-Oliger")
    ap.add_argument("--sigma", type=float, default=0.01, help="Kreiss-Oliger sigma (fd6)")
    args = ap.parse_args(argv)

    wl = I.EXTREMAL_GRAV_HYP.with_(nr=args.nr, nth=args.nth, wprec=args.wprec)
    scheme = TEUK_SCHEME_FD6_KO8 if args.scheme == "fd6" else TEUK_SCHEME_WENO5
    h = teuk_create(params_from_workload(wl, scheme=scheme, ko_sigma=args.sigma))
    teuk_set_state(h, I.initial_data(wl), 0.0)
    _, dt, _ = teuk_get_info(h)
    total = args.steps if args.steps > 0 else int(np.ceil(args.tau / dt))
    chunk = max(1, min(total, int(round(args.every / dt))))
    j = wl.nth // 2
    label = f"FD6 + KO8 (sigma {args.sigma:g})" if args.scheme == "fd6" else f"weights {wl.wprec}"
    print(f"# {wl.name}: {wl.nr} x {wl.nth}, {label}, dt = {dt:.6g} M, {total} steps")
    print("#      tau        Phi_H     dPhi_H/drho     Phi_scri    p(Phi_H)")
    done, prev, stepping = 0, None, 0.0
    while done < total:
        n = min(chunk, total - done)
        t0 = time.perf_counter()
        teuk_step(h, n)
        wave, hor, tau = teuk_observe(h, wl.S)        # synchronises the stream
        stepping += time.perf_counter() - t0
        done += n
        phi = hor[j, 0]
        p = tau * (phi - prev[1]) / (tau - prev[0]) / phi if prev else float("nan")
        print(f"{tau:10.3f} {phi:12.5e} {hor[j, 4]:14.5e} {wave[j, 0]:12.5e} {p:10.3f}")
        prev = (tau, phi)
    h.close()
    rate = wl.nr * wl.nth * 3 * total / stepping
    print(f"# {rate:.4g} point-stage updates/s over {total} steps (observation included)")


if __name__ == "__main__":
    main()
