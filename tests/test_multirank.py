"""The N > 1 host path of bench.py on CPU: two gloo ranks, the barrier, the
max over ranks of the timed region and the whole-job (weak-scaling) value."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    my_ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
    mx = bench.max_over_ranks(my_ms, w, torch.device("cpu"))
    value = bench.weak_scaling_value(1000, 4, w, mx)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as fh:
        json.dump({"max_ms": mx, "value": value}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_value(tmp_path):
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["max_ms"] == 15.0
        assert abs(r["value"] - 1000 * 4 * 2 / 0.015) < 1e-6


REQUIRED = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
            "cpu_baseline", "e2e"}


def _json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one
    JSON line with the contract's keys, for the benchmark's metric and
    workload, with no host-device bytes."""
    import subprocess
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    lines = _json_lines(out.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert REQUIRED <= set(d), REQUIRED - set(d)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.WL.name


def test_reference_arm_under_torchrun_prints_from_rank_0_only():
    """With two ranks (gloo on CPU) rank 0 alone runs the oracle and prints;
    the other rank exits 0 without work."""
    import subprocess
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def _rank_failing(rank, world, port, outdir):
    """Rank 1 leaves before the barrier (between steps, nothing in flight);
    rank 0 must learn of it from the collective, within the group timeout."""
    import time
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), TEUK_PG_TIMEOUT_S="20")
    sys.path.insert(0, ROOT)
    import bench
    bench.dist_init(world)
    if rank == 1:
        os._exit(0)
    t0 = time.time()
    try:
        bench.barrier(world)
        bench.max_over_ranks(1.0, world, torch.device("cpu"))
        outcome = "completed"
    except Exception as e:                                  # noqa: BLE001
        outcome = "raised: " + type(e).__name__
    with open(os.path.join(outdir, "rank0.json"), "w") as fh:
        json.dump({"outcome": outcome, "seconds": time.time() - t0}, fh)
    os._exit(0)


def test_a_rank_that_leaves_ends_the_others_collective_with_an_error(tmp_path):
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [mp.Process(target=_rank_failing, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = json.load(open(tmp_path / "rank0.json"))
    assert res["outcome"].startswith("raised"), res
    assert res["seconds"] < 60, res

