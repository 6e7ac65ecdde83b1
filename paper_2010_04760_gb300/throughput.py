"""Throughput of the named workloads, per weight format, on cuda:0.

    python -m paper_2010_04760_gb300.throughput [--steps 20] [--per-call K]
        [--workload NAME] [--wprec FMT] [--launch auto|stages|fused]

For each workload and weight format: point-stage updates per second (nodes x
stages per step: 3 for SSP-RK(3,3), 10 for SSP-RK(10,4)), device-timed with
CUDA events around each teuk_step call through a handle (one step per call
unless --per-call), L2 flushed before every call by writing a 256 MiB
buffer, as the benchmark does; the last column says whether teuk_step ran
the fused persistent step or stage launches; the HBM figure divides the algorithmic bytes of a point-stage
(coefficient planes, u_prev, u_out and, for SSP-RK(3,3), 2/3 of u^n) by the
time, and "M/s" is simulated time (units of M) advanced per second. The last
rows run the paper's comparison scheme (FD6 + KO8, Sec. 3.1.1) and its
second integrator (SSP-RK(10,4), Sec. 3.2). Prints one table row per case.
"""
import argparse

import numpy as np

from . import inputs as I
from . import (TEUK_LAUNCH_FUSED, TEUK_LAUNCH_STAGES, TEUK_RK_SSP104, TEUK_SCHEME_FD6_KO8,
               params_from_workload, teuk_create, teuk_get_info, teuk_get_launch,
               teuk_set_launch, teuk_set_state, teuk_step)

FD6 = {"scheme": TEUK_SCHEME_FD6_KO8}
RK104 = {"rk": TEUK_RK_SSP104}
# (workload, weight formats, parameter overrides, label)
CASES = [
    (I.SCHW_SCALAR, ("fp64", "fp32"), {}, ""),
    (I.KERR_GRAV, ("fp64", "fp32", "fp16", "bf16"), {}, ""),
    (I.EXTREMAL_SCALAR, ("fp64", "fp32", "fp16", "bf16"), {}, ""),
    (I.TAIL_SCALAR, ("fp64", "fp32"), {}, ""),
    (I.EXTREMAL_GRAV_HYP, ("fp64", "fp32", "fp16", "bf16"), {}, ""),
    (I.KERR_GRAV, ("fp64",), FD6, " FD6+KO8"),
    (I.EXTREMAL_GRAV_HYP, ("fp64",), FD6, " FD6+KO8"),
    (I.KERR_GRAV, ("fp64", "fp32"), RK104, " RK(10,4)"),
    (I.EXTREMAL_GRAV_HYP, ("fp64", "fp32"), RK104, " RK(10,4)"),
]


def bytes_per_point_stage(wl, rk104=False):
    """Coefficients, u_prev, u_out, plus: SSP-RK(3,3) reads u^n in two of its
    three stages; SSP-RK(10,4) reads q in its last stage and its combination
    kernel reads two states and writes two (160 B per node per ten stages)."""
    planes = 12 if wl.coords == 1 else 11        # the kernel reads 12 of the 13 planes
    return 8.0 * planes + 32.0 + 32.0 + (16.0 if rk104 else 32.0 * 2.0 / 3.0)


def time_case(torch, wl, wprec, steps, stream, flush, over=None, launch=None, per_call=1):
    """Device time per step, `steps` calls of teuk_step(h, per_call), the L2
    flushed before each call. Returns (rate, ms/step, GB/s, M/s, fused)."""
    over = over or {}
    rk104 = over.get("rk") == TEUK_RK_SSP104
    stages = 10 if rk104 else 3
    h = teuk_create(params_from_workload(wl, wprec=wprec, **over), stream)
    if launch is not None:
        teuk_set_launch(h, launch)
    fused = teuk_get_launch(h)[2] == 1
    _, dt, _ = teuk_get_info(h)
    teuk_set_state(h, I.initial_data(wl), 0.0)
    for _ in range(3):
        teuk_step(h, per_call)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(k & 255)
            ev[k][0].record(stream)
            teuk_step(h, per_call)
            ev[k][1].record(stream)
    stream.synchronize()
    h.close()
    ms = np.mean([a.elapsed_time(b) for a, b in ev]) / per_call
    rate = wl.nr * wl.nth * stages / (ms * 1e-3)
    return rate, ms, rate * bytes_per_point_stage(wl, rk104) / 1e9, dt / (ms * 1e-3), fused


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=20, help="timed teuk_step calls per case")
    ap.add_argument("--per-call", type=int, default=1, help="steps per teuk_step call")
    ap.add_argument("--workload", default=None, help="only workloads whose name contains this")
    ap.add_argument("--wprec", default=None, help="only this weight format")
    ap.add_argument("--launch", choices=["auto", "stages", "fused"], default="auto")
    args = ap.parse_args(argv)
    launch = {"auto": None, "stages": TEUK_LAUNCH_STAGES, "fused": TEUK_LAUNCH_FUSED}[args.launch]
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    print(f"{'workload':44s} {'weights':7s} {'pt-stage/s':>11s} {'ms/step':>9s} {'HBM GB/s':>9s}"
          f" {'M/s':>9s} launch")
    for wl, formats, over, label in CASES:
        if args.workload and args.workload not in wl.name:
            continue
        for wprec in formats:
            if args.wprec and wprec != args.wprec:
                continue
            lo = launch if (over.get("rk", 0) == 0 and over.get("scheme", 0) == 0) else None
            rate, ms, gbs, mps, fused = time_case(torch, wl, wprec, args.steps, stream, flush,
                                                  over, lo, args.per_call)
            print(f"{wl.name + label:44s} {wprec:7s} {rate:11.4g} {ms:9.4f} {gbs:9.1f} {mps:9.1f} "
                  f"{'fused' if fused else 'stages'}", flush=True)


if __name__ == "__main__":
    main()
