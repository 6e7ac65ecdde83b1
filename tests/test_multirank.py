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
