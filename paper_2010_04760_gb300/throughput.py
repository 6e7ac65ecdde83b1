"""Throughput of the named workloads, per weight format, on cuda:0.

    python -m paper_2010_04760_gb300.throughput [--steps 20]

For each workload and weight format: point-stage updates per second (nodes x 3
stages per SSP-RK(3,3) step), device-timed with CUDA events around each step
through a handle (one teuk_step call per step), L2 flushed before every step
by writing a 256 MiB buffer, as the benchmark does; the HBM figure divides
the algorithmic bytes of a point-stage (coefficient planes, u_prev, u_out and
2/3 of u^n) by the time. Prints one table row per case.
"""
import argparse

import numpy as np

from . import inputs as I
from . import params_from_workload, teuk_create, teuk_set_state, teuk_step

CASES = [
    (I.SCHW_SCALAR, ("fp64", "fp32")),
    (I.KERR_GRAV, ("fp64", "fp32", "fp16", "bf16")),
    (I.EXTREMAL_SCALAR, ("fp64", "fp32", "fp16", "bf16")),
    (I.TAIL_SCALAR, ("fp64", "fp32")),
    (I.EXTREMAL_GRAV_HYP, ("fp64", "fp32", "fp16", "bf16")),
]


def bytes_per_point_stage(wl):
    planes = 12 if wl.coords == 1 else 11        # the kernel reads 12 of the 13 planes
    return 8.0 * planes + 32.0 + 32.0 + 32.0 * 2.0 / 3.0


def time_case(torch, wl, wprec, steps, stream, flush):
    h = teuk_create(params_from_workload(wl, wprec=wprec), stream)
    teuk_set_state(h, I.initial_data(wl), 0.0)
    for _ in range(3):
        teuk_step(h, 1)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(k & 255)
            ev[k][0].record(stream)
            teuk_step(h, 1)
            ev[k][1].record(stream)
    stream.synchronize()
    h.close()
    ms = np.mean([a.elapsed_time(b) for a, b in ev])
    rate = wl.nr * wl.nth * 3 / (ms * 1e-3)
    return rate, ms, rate * bytes_per_point_stage(wl) / 1e9


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=20)
    args = ap.parse_args(argv)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    print(f"{'workload':34s} {'weights':7s} {'pt-stage/s':>11s} {'ms/step':>9s} {'HBM GB/s':>9s}")
    for wl, formats in CASES:
        for wprec in formats:
            rate, ms, gbs = time_case(torch, wl, wprec, args.steps, stream, flush)
            print(f"{wl.name:34s} {wprec:7s} {rate:11.4g} {ms:9.4f} {gbs:9.1f}", flush=True)


if __name__ == "__main__":
    main()
