"""Benchmark: WENO5 Teukolsky point-stage updates/s, mixed vs binary64 weights.

Workload: the near-extremal gravitational evolution, Kerr a = 0.999 M,
s = -2, m = 2, grid 2048 (r* in [-100, 300] M) x 128 (theta), seeded Gaussian
l = 2 pulse at r* = 30 M (width 3 M). A step is one SSP-RK(3,3) step: three
fused stage launches over all 262,144 nodes (786,432 point-stage updates).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Timing: W untimed warm-up steps, then K timed steps; before each timed step a
256 MiB buffer is written to flush the 129 MB L2 (the workload's state and
coefficients, ~50 MB, would otherwise stay L2-resident), and each step is
bracketed by CUDA events on the launching stream. Max over ranks. With N > 1
(torchrun) every rank evolves its own replica (no data exchange; weak scaling).
The reference arm (--impl reference) times the CPU oracle on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2010_04760_gb300 import inputs as I  # noqa: E402

WL = I.KERR_GRAV
METRIC = "WENO5 Teukolsky point-stage updates/s, mixed vs FP64 weights, at stated L2 err"
UNIT = "point-stage updates/s"
POINTS = WL.nr * WL.nth
# binary64 flops per point-stage of the fused stage (FMA = 2), averaged over
# the three SSP-RK(3,3) stages: first differences 4, third differences 12,
# weighted fluxes 24, derivatives 12, Psi rows 8, pi rows 44; the second stage,
# kept as 4 u^(2), folds 3 u^n into the rows (+4 and +4), the third adds the
# combination alpha u^n + beta (...) (12) -> (104 + 112 + 116) / 3.
FP64_FLOPS_PER_PT_STAGE = (104.0 + 112.0 + 116.0) / 3.0
# algorithmic HBM bytes per point-stage: 11 coefficient planes (88 B), u_prev
# (32 B), u_out (32 B), u^n in stages 2 and 3 (2/3 x 32 B).
BYTES_PER_PT_STAGE = 88.0 + 32.0 + 32.0 + 32.0 * 2.0 / 3.0
# DRAM bytes (read + write) per launch of the binary32-weight kernel on this
# workload, from one ncu capture on these kernel sources: the fused step kernel
# (one launch = one step), averaged over three launches; valid only for the
# sources it was taken on, identified by the sha256 of their concatenation.
NCU_TRAFFIC = {"sources": ["paper_2010_04760_gb300/csrc/teuk_stage_kernels.cuh",
                           "paper_2010_04760_gb300/csrc/teuk_stage.cu"],
               "sha256": "8f707ed7140000abda869bfac7c57a7e66cadbd2f78163b16bd1f1cae006ad7a",
               "bytes_per_launch": None,
               "fused_bytes_per_launch": (31525376 + 5632 + 31525632 + 22784 + 31526144
                                          + 11008) / 3.0}


def workload_config(wl, wprec):
    """The `config` object of both arms' JSON lines."""
    return {"workload": wl.name, "nr": wl.nr, "ntheta": wl.nth, "a": wl.a, "s": wl.s,
            "m": wl.m, "wprec": wprec, "rk": "SSP-RK(3,3)"}


def kernel_source_digest(sources=None):
    import hashlib
    h = hashlib.sha256()
    for rel in sources or NCU_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(fused=False):
    try:
        digest = kernel_source_digest()
    except OSError:
        return None
    if digest != NCU_TRAFFIC["sha256"]:
        return None
    return NCU_TRAFFIC["fused_bytes_per_launch" if fused else "bytes_per_launch"]


# Binary64 FMA lanes per SM per clock on GB300 (its nominal 1.26 TFLOP/s =
# 152 SMs x 2 lanes x 2 flops x 2.07 GHz). The roofline peak is derived from
# this, the device's SM count and the SM clock sampled in the timed region.
FP64_FMA_LANES_PER_SM_CLK = 2
SM_MAX_MHZ = 2070.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[3:]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_init(gpus):
    """Rank and world size from the torchrun environment; one process group
    (NCCL on GPUs, gloo without) used only for the barrier and the max over
    ranks of the timed region: the replicas exchange no data."""
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import datetime
        import torch
        import torch.distributed as dist
        # a rank that dies or never arrives ends the others' next collective
        # with an error after this long instead of the library default (30 min)
        timeout = datetime.timedelta(seconds=float(os.environ.get("TEUK_PG_TIMEOUT_S", "600")))
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo", timeout=timeout)
    return rank, world


def weak_scaling_value(points_per_step, steps, world, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return points_per_step * steps * world / (max_ms * 1e-3)


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def time_gpu_steps(T, torch, wprec, steps, warmup, stream, flush, launch=None):
    """Device time of `steps` RK steps of the workload with weights `wprec`
    (launch: a teuk_launch mode, default the library's choice)."""
    p = T.params_from_workload(WL, wprec=wprec)
    h = T.teuk_create(p, stream)
    if launch is not None:
        T.teuk_set_launch(h, launch)
    time_gpu_steps.launch_used = "fused" if T.teuk_get_launch(h)[2] == 1 else "stages"
    T.teuk_set_state(h, I.initial_data(WL), 0.0)
    for _ in range(warmup):
        T.teuk_step(h, 1)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.nvtx.range_push(f"{wprec}_timed" + ("" if launch is None else f"_launch{launch}"))
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(float(k))                 # write > L2 between timed steps
            ev[k][0].record(stream)
            T.teuk_step(h, 1)
            ev[k][1].record(stream)
    stream.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = [a.elapsed_time(b) for a, b in ev]
    assert T.teuk_check_finite(h) == T.TEUK_OK
    h.close()
    return sum(ms), ms


def waveform_error(T, torch, stream, t_end=WL.t_end, r_ext=50.0):
    """Relative L2 difference of the waveform (Psi at r* = r_ext over all theta,
    sampled every 100 steps up to t_end, the workload's stated duration of
    500 M) between each reduced weight format and binary64 weights."""
    waves = {}
    t = 0.0
    for wprec in ("fp64", "fp32", "fp16", "bf16"):
        h = T.teuk_create(T.params_from_workload(WL, wprec=wprec), stream)
        T.teuk_set_state(h, I.initial_data(WL), 0.0)
        _, dt, _ = T.teuk_get_info(h)
        ws = []
        for _ in range(max(1, int(t_end / dt) // 100)):
            T.teuk_step(h, 100)
            ws.append(T.teuk_observe(h, r_ext)[0].copy())
        _, dt, t = T.teuk_get_info(h)
        h.close()
        waves[wprec] = np.array(ws)
    ref = np.linalg.norm(waves["fp64"])
    errs = {w: float(np.linalg.norm(waves[w] - waves["fp64"]) / ref) for w in ("fp32", "fp16", "bf16")}
    return errs, t


def time_multi_step(T, torch, wprec, steps, warmup, stream, flush):
    """Device time of `steps` RK steps issued as one teuk_step call (the way a
    long evolution runs), L2 flushed before the call."""
    p = T.params_from_workload(WL, wprec=wprec)
    h = T.teuk_create(p, stream)
    T.teuk_set_state(h, I.initial_data(WL), 0.0)
    T.teuk_step(h, max(warmup, 4))
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(f"{wprec}_multi_timed")
    with torch.cuda.stream(stream):
        flush.fill_(1)
        e0.record(stream)
        T.teuk_step(h, steps)
        e1.record(stream)
    stream.synchronize()
    torch.cuda.nvtx.range_pop()
    assert T.teuk_check_finite(h) == T.TEUK_OK
    h.close()
    return e0.elapsed_time(e1)


def time_e2e(T, torch, steps, warmup, stream, flush):
    """The metric end to end through the public handle API with host buffers,
    timed like the device value: one handle on the bench stream, L2 flushed
    before every step (outside the timed region), and per step CUDA events
    around the upload of the step's input state from pinned host memory
    (teuk_set_state_async), one RK step (teuk_step) and the read-back of its
    result into pinned host memory (teuk_get_state_async)."""
    p = T.params_from_workload(WL)
    h = T.teuk_create(p, stream)
    src = torch.empty((4, WL.nth, WL.nr), dtype=torch.float64, pin_memory=True).numpy()
    src[...] = I.initial_data(WL)
    dst = torch.empty((4, WL.nth, WL.nr), dtype=torch.float64, pin_memory=True).numpy()
    for _ in range(warmup):
        T.teuk_set_state_async(h, src, 0.0)
        T.teuk_step(h, 1)
        T.teuk_get_state_async(h, dst)
    T.teuk_synchronize(h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            T.teuk_set_state_async(h, src, 0.0)
            T.teuk_step(h, 1)
            T.teuk_get_state_async(h, dst)
            ev[k][1].record(stream)
    T.teuk_synchronize(h)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ok = bool(np.isfinite(dst).all())
    h.close()
    return ms, src.nbytes, ok


def time_e2e_pipelined(T, torch, steps, lanes=3):
    """Independent problems pipelined over `lanes` handles, each on its own
    stream: one problem's copies overlap another's stepping, and the streams'
    kernels may run concurrently; no L2 flush. Wall-clock seconds."""
    p = T.params_from_workload(WL)
    hs = [T.teuk_create(p) for _ in range(lanes)]
    ins, outs = [], []
    for _ in range(lanes):
        a = torch.empty((4, WL.nth, WL.nr), dtype=torch.float64, pin_memory=True).numpy()
        a[...] = I.initial_data(WL)
        ins.append(a)
        outs.append(torch.empty((4, WL.nth, WL.nr), dtype=torch.float64, pin_memory=True).numpy())

    def run(n):
        for i in range(n):
            k = i % lanes
            if i >= lanes:
                T.teuk_synchronize(hs[k])          # its previous result has landed
            T.teuk_set_state_async(hs[k], ins[k], 0.0)
            T.teuk_step(hs[k], 1)
            T.teuk_get_state_async(hs[k], outs[k])
        for h in hs:
            T.teuk_synchronize(h)

    run(2 * lanes)                                 # warm-up (graphs, pages)
    t0 = time.perf_counter()
    run(steps)
    el = time.perf_counter() - t0
    for h in hs:
        h.close()
    return el


def time_workload(T, torch, wl, wprec, steps, warmup, stream, flush, fp64_peak_derived):
    """Device time per RK step of workload wl with weights wprec (L2 flushed
    before every step), its throughput and its binary64-pipe fraction."""
    p = T.params_from_workload(wl, wprec=wprec)
    h = T.teuk_create(p, stream)
    T.teuk_set_state(h, I.initial_data(wl), 0.0)
    for _ in range(warmup):
        T.teuk_step(h, 1)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            T.teuk_step(h, 1)
            ev[k][1].record(stream)
    stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    finite = T.teuk_check_finite(h) == T.TEUK_OK
    h.close()
    pts = wl.nr * wl.nth
    rate = pts * 3 / (ms * 1e-3)
    out = {"value": rate, "unit": UNIT, "ms_per_step": ms, "steps": steps, "finite": finite}
    if wprec != "fp64":
        tf = FP64_FLOPS_PER_PT_STAGE * rate / 1e12
        out["fp64_tflops"] = tf
        out["fp64_frac"] = tf / fp64_peak_derived
        out["hbm_gbs"] = BYTES_PER_PT_STAGE * rate / 1e9
    return out


def time_batch(T, torch, stream, steps=32):
    """Throughput of the 64-member uneven batch (one persistent launch per RK
    stage over all members, graph-replayed; ~43 M nodes, state and
    coefficients ~7.8 GB, far larger than L2)."""
    wls = I.batch_workloads()
    ps = [T.params_from_workload(w) for w in wls]
    b = T.teuk_batch_create(ps, stream, autotune=True)
    for k, w in enumerate(wls):
        T.teuk_batch_set_state(b, k, I.initial_data(w), 0.0)
    T.teuk_batch_step(b, 16)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    T.teuk_batch_step(b, steps)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    _, _, seg, ctas = T.teuk_batch_get_info(b, 0)
    b.close()
    nodes = sum(w.nr * w.nth for w in wls)
    return {"value": nodes * 3 * steps / (ms * 1e-3), "unit": UNIT, "members": len(wls),
            "nodes": nodes, "steps": steps, "ms_per_step": ms / steps, "segment": seg,
            "ctas_per_sm": ctas, "wprec": "fp32"}


def time_paper_run(T, torch, stream, steps=200):
    """Throughput on the paper's own run (Sec. 4): 16384 (rho) x 64 (theta)
    on the hyperboloidal slices, extremal Kerr, s = -2, (l, m) = (2, 0),
    binary32 weights; state and 13 coefficient planes ~143 MB, above L2."""
    wl = I.EXTREMAL_GRAV_HYP
    h = T.teuk_create(T.params_from_workload(wl), stream)
    T.teuk_set_state(h, I.initial_data(wl), 0.0)
    T.teuk_step(h, 32)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    T.teuk_step(h, steps)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    st = T.teuk_check_finite(h)
    h.close()
    return {"value": wl.nr * wl.nth * 3 * steps / (ms * 1e-3), "unit": UNIT,
            "workload": wl.name, "steps": steps, "ms_per_step": ms / steps, "wprec": wl.wprec,
            "finite": st == T.TEUK_OK}


def oracle_rate(nsteps_budget_s=15.0, wprec="fp32", max_steps=1000):
    """Oracle point-stage updates/s on the workload, over a bounded number of
    RK steps chosen to take about nsteps_budget_s seconds."""
    import oracle as o
    g = o.grid(WL.nr, WL.nth, WL.rs_min, WL.rs_max, WL.M, WL.a, WL.s, WL.m, WL.eps, wprec)
    co = o.coefficients(g)
    u = I.initial_data(WL)
    dt = 0.005
    t0 = time.perf_counter()
    u = o.rk3_step(g, co, dt, u, 1)
    t1 = time.perf_counter() - t0
    n = int(max(2, min(max_steps, nsteps_budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    u = o.rk3_step(g, co, dt, u, n)
    el = time.perf_counter() - t0
    return POINTS * 3 * n / el, n, el, o.num_threads()


def run_reference(args, rank, world):
    """The CPU oracle on the host cores, one SSP-RK(3,3) step of the workload
    per timed step (rank 0 only)."""
    if rank != 0:
        return
    import oracle as o
    o.build()
    g = o.grid(WL.nr, WL.nth, WL.rs_min, WL.rs_max, WL.M, WL.a, WL.s, WL.m, WL.eps, "fp32")
    co = o.coefficients(g)
    u = I.initial_data(WL)
    dt = 0.005
    u = o.rk3_step(g, co, dt, u, args.warmup)
    t0 = time.perf_counter()
    u = o.rk3_step(g, co, dt, u, args.steps)
    el = time.perf_counter() - t0
    value = POINTS * 3 * args.steps / el
    cores = o.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "weights_dtype": "f32",
            "data": "synthetic",
            "config": {**workload_config(WL, "fp32"),
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": "replicas x1"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} RK steps of the {WL.nr}x{WL.nth} workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_2010_04760_gb300 as T
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    T.lib()
    stream = torch.cuda.Stream(device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    # clocks sampled over every device-timed region of the workload (the
    # binary64-weight baseline, the headline, the stage-launch comparison and
    # the end-to-end run)
    with ClockSampler(local) as clk:
        # binary64-weight baseline on the same workload
        barrier(world)
        ms64, _ = time_gpu_steps(T, torch, "fp64", args.steps, args.warmup, stream, flush)
        ms64 = max_over_ranks(ms64, world, device)
        # mixed precision (binary32 weights): the headline
        barrier(world)
        ms32, per = time_gpu_steps(T, torch, "fp32", args.steps, args.warmup, stream, flush)
        ms32 = max_over_ranks(ms32, world, device)
        launch32 = time_gpu_steps.launch_used
        # the same, one step per call, with the other schedule
        other_launch = T.TEUK_LAUNCH_FUSED if launch32 == "stages" else T.TEUK_LAUNCH_STAGES
        barrier(world)
        ms32s, _ = time_gpu_steps(T, torch, "fp32", args.steps, args.warmup, stream, flush,
                                  other_launch)
        ms32s = max_over_ranks(ms32s, world, device)
        # all K steps in one teuk_step call (the fused step: one persistent
        # launch), L2 flushed once before
        barrier(world)
        ms32m = time_multi_step(T, torch, "fp32", args.steps, args.warmup, stream, flush)
        ms32m = max_over_ranks(ms32m, world, device)
        barrier(world)
        e2e_ms, nbytes, e2e_ok = time_e2e(T, torch, args.steps, args.warmup, stream, flush)
        e2e_ms = max_over_ranks(e2e_ms, world, device)
    pipe_steps = max(60, args.steps)
    pipe_s = max_over_ranks(time_e2e_pipelined(T, torch, pipe_steps), world, device)
    err, t_err = waveform_error(T, torch, stream) if rank == 0 else (None, None)
    batch = time_batch(T, torch, stream) if rank == 0 else None
    paper_run = time_paper_run(T, torch, stream) if rank == 0 else None

    fp64_peak_tf = 2.0 * T.teuk_fp64_fma_rate(stream) / 1e12      # measured live
    clk_summary = clk.summary()
    sm_clock_mhz = clk_summary.get("sm_mhz") or SM_MAX_MHZ
    SMS = torch.cuda.get_device_properties(device).multi_processor_count
    fp64_peak_derived = SMS * FP64_FMA_LANES_PER_SM_CLK * 2 * sm_clock_mhz * 1e6 / 1e12
    value = weak_scaling_value(POINTS * 3, args.steps, world, ms32)
    value64 = weak_scaling_value(POINTS * 3, args.steps, world, ms64)
    fused = launch32 == "fused"
    launch_ms = ms32 / (3 * args.steps)          # per stage
    achieved_tf = FP64_FLOPS_PER_PT_STAGE * POINTS / (launch_ms * 1e-3) / 1e12
    achieved_gbs = BYTES_PER_PT_STAGE * POINTS / (launch_ms * 1e-3) / 1e9
    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if rank != 0:
        return
    # the other large workloads: the extremal scalar 8192 x 256 with binary16
    # and bfloat16 weights, the tail workload 16384 x 512 with binary32, each
    # beside binary64 weights (device-timed per step, L2 flushed as above)
    other = {}
    for wl, formats in ((I.EXTREMAL_SCALAR, ("fp64", "fp16", "bf16")),
                        (I.TAIL_SCALAR, ("fp64", "fp32"))):
        rows = {w: time_workload(T, torch, wl, w, 10, 3, stream, flush, fp64_peak_derived)
                for w in formats}
        for w in formats[1:]:
            rows[w]["speedup_vs_fp64_weights"] = rows[w]["value"] / rows["fp64"]["value"]
        other[wl.name] = {"config": workload_config(wl, formats[1]), **rows}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "weights_dtype": "f32",
        "data": "synthetic",
        "config": {**workload_config(WL, "fp32"),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "launch": ("fused step (one persistent launch per step)" if fused
                   else "three stage launches per step (programmatic dependent launch)"),
        "other_launch_per_step": {
            "value": weak_scaling_value(POINTS * 3, args.steps, world, ms32s),
            "ms_per_step": ms32s / args.steps,
            "how": ("the same, one step per call, as " +
                    ("three stage launches" if fused else "one fused persistent launch"))},
        "one_call_of_k_steps": {
            "value": weak_scaling_value(POINTS * 3, args.steps, world, ms32m),
            "ms_per_step": ms32m / args.steps,
            "how": f"the same {args.steps} steps as one teuk_step call: one fused persistent "
                   "launch (up to 1024 steps), L2 flushed once before; how a long evolution "
                   "runs (the state stays L2-resident between steps)"},
        "fp64_weights": {"value": value64, "ms_per_step": ms64 / args.steps},
        "mixed_speedup_vs_fp64_weights": value / value64,
        "paper_mixed_speedup_context": {
            "value": 3.3, "what": "binary128 state with binary64 weights vs all-binary128, "
            "WENO5 in rho, 16384 x 64 (Sec. 4-5)", "hardware": "not stated in the paper "
            "(its GPU runs use V100 nodes)", "comparable": False},
        "waveform_rel_l2_fp32_vs_fp64_weights": err["fp32"],
        "waveform_rel_l2_vs_fp64_weights": err,
        "waveform_error_window": f"Psi(r*=50M, all theta) every 100 steps to t={t_err:.1f}M",
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak_derived,
                     "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak_derived,
                     "traffic": ncu_traffic(fused), "traffic_unit": "bytes per launch",
                     "algorithmic_bytes_per_launch":
                         BYTES_PER_PT_STAGE * POINTS * (3 if fused else 1),
                     "pipe": "fp64",
                     "peak_source": f"derived: {SMS} SMs x {FP64_FMA_LANES_PER_SM_CLK} binary64 "
                                    f"FMA lanes/clk x 2 flops x {sm_clock_mhz:.0f} MHz "
                                    "(median SM clock sampled during the timed region)",
                     "measured_sustained_peak": fp64_peak_tf,
                     "frac_of_measured_sustained": achieved_tf / fp64_peak_tf,
                     "measured_source": "teuk_fp64_fma_rate: independent binary64 FMA "
                                        "chains on this GPU, x2 flops",
                     "kernel": ("fused_step_kernel<fp32 weights> (one launch = one step "
                                "= 3 stages)") if fused else "stage_kernel<fp32 weights>",
                     "flops_per_point_stage": FP64_FLOPS_PER_PT_STAGE},
        "roofline_hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gbs / hbm_peak,
                         "bytes_per_point_stage": BYTES_PER_PT_STAGE},
        "e2e": {"value": weak_scaling_value(POINTS * 3, args.steps, world, e2e_ms),
                "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "steps": args.steps, "ms_per_step": e2e_ms / args.steps, "finite": e2e_ok,
                "how": "per step, timed with CUDA events on one handle's stream after an L2 "
                       "flush: teuk_set_state_async from pinned host memory, teuk_step(1), "
                       "teuk_get_state_async to pinned host memory (the device value's step "
                       "plus both copies)"},
        "e2e_pipelined_3_handles": {
            "value": POINTS * 3 * pipe_steps * world / pipe_s, "unit": UNIT,
            "steps": pipe_steps, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "how": "independent steps over 3 handles on 3 streams with the asynchronous copy "
                   "calls (one problem's copies overlap another's step, kernels of different "
                   "streams may run concurrently), wall clock, no L2 flush"},
        "other_workloads": other,
        "batched_64_uneven_evolutions": batch,
        "paper_run_hyperboloidal_16384x64": paper_run,
        "gpu_launches": (1 if fused else 3) * args.steps,
        "clocks": clk.summary(),
    }
    v, n, el, cores = oracle_rate()
    line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n} RK steps of the {WL.nr}x{WL.nth} workload "
                                          f"(binary32 weights), {el:.1f} s"}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
