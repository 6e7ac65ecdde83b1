"""The radial slab decomposition of the paper's MPI runs (Sec. 4.1) on CPU
ranks: two gloo ranks each hold one r* slab of the grid with three halo nodes
on the inner side, evolve it with the oracle's right-hand side through the
printed SSP-RK(3,3) stages, and after every stage send their three edge
columns to the other rank, which writes them into its halo. The grid's nodes
are whole numbers of M (spacing exactly 1), so a slab's own grid, spacing and
coefficients are those of the undivided grid bit for bit, and each rank's
interior must equal the undivided evolution bit for bit. A run without the
exchange shows that the halos matter."""
import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HALO = 3
NR, NTH, RS0 = 160, 8, -60.0          # r* = -60 .. 99 M, one node per M
CUT = 83                              # rank 0 holds nodes [0, 83), rank 1 [83, 160)
STEPS, DT = 15, 0.2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grid(o, lo, hi):
    """The oracle grid of nodes lo .. hi-1 of the undivided grid."""
    return o.grid(hi - lo, NTH, RS0 + lo, RS0 + hi - 1, 1.0, 0.9, -2, 2)


def _step(o, g, co, u, exchange):
    """One printed SSP-RK(3,3) step (Sec. 3.2) with `exchange` after every stage."""
    u1 = u + DT * o.rhs(g, co, u)
    exchange(u1)
    u2 = 0.75 * u + 0.25 * (u1 + DT * o.rhs(g, co, u1))
    exchange(u2)
    u3 = u / 3.0 + 2.0 / 3.0 * (u2 + DT * o.rhs(g, co, u2))
    exchange(u3)
    return u3


def _initial(o):
    sys.path.insert(0, ROOT)
    from paper_2010_04760_gb300 import inputs as I
    wl = I.KERR_GRAV.with_(nr=NR, nth=NTH, rs_min=RS0, rs_max=RS0 + NR - 1, rc=15.0)
    return I.initial_data(wl)


def _rank_main(rank, world, port, outdir, do_exchange):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import oracle as o
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u0 = _initial(o)
    # rank 0: interior [0, CUT), halo [CUT, CUT+3); rank 1: halo [CUT-3, CUT), interior [CUT, NR)
    lo, hi = (0, CUT + HALO) if rank == 0 else (CUT - HALO, NR)
    g = _grid(o, lo, hi)
    co = o.coefficients(g)
    u = u0[..., lo:hi].copy()
    peer = 1 - rank

    def exchange(v):
        if not do_exchange:
            return
        if rank == 0:
            send = np.ascontiguousarray(v[..., CUT - HALO:CUT])          # last interior nodes
            recv_into = (slice(None), slice(None), slice(CUT, CUT + HALO))
        else:
            send = np.ascontiguousarray(v[..., HALO:2 * HALO])          # first interior nodes
            recv_into = (slice(None), slice(None), slice(0, HALO))
        buf = torch.empty(send.shape, dtype=torch.float64)
        reqs = [dist.isend(torch.from_numpy(send), peer), dist.irecv(buf, peer)]
        for r in reqs:
            r.wait()
        v[recv_into] = buf.numpy()

    for _ in range(STEPS):
        u = _step(o, g, co, u, exchange)
    # the undivided evolution, computed by each rank for itself
    gf = _grid(o, 0, NR)
    cf = o.coefficients(gf)
    uf = u0.copy()
    for _ in range(STEPS):
        uf = _step(o, gf, cf, uf, lambda v: None)
    mine = u[..., :CUT] if rank == 0 else u[..., HALO:]
    ref = uf[..., :CUT] if rank == 0 else uf[..., CUT:]
    with open(os.path.join(outdir, f"slab{rank}.json"), "w") as fh:
        json.dump({"equal": bool(np.array_equal(mine, ref)),
                   "max_diff": float(np.max(np.abs(mine - ref)))}, fh)
    dist.barrier()
    dist.destroy_process_group()


def _run(tmp_path, do_exchange):
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, str(tmp_path), do_exchange))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return [json.load(open(tmp_path / f"slab{r}.json")) for r in range(2)]


def test_two_rank_slabs_with_halo_exchange_are_exact(tmp_path):
    res = _run(tmp_path, True)
    assert all(r["equal"] for r in res), res


def test_slabs_without_the_exchange_diverge(tmp_path):
    res = _run(tmp_path, False)
    assert any(r["max_diff"] > 1e-6 for r in res), res
