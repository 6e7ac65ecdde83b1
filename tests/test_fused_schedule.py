"""Host-side model of the fused step kernel's schedule (teuk_stage_kernels.cuh,
fused_step_kernel): tickets t = epoch * items + item handed out in order, each
block taking its next ticket as soon as it starts the current one, an item of
epoch e starting once its 3 x 3 neighbourhood of items has completed epoch
e - 1. A discrete-event simulation with random item durations checks the
claim the kernel rests on: every read of a buffer (the radial and theta
stencils reach only the neighbouring items) starts after the write it needs
has finished, and no write of a buffer starts before the reads of the value
it replaces have finished (stage 1 writes w1 and reads u around the item,
stage 2 writes w2 and reads w1 around it and u at the item, stage 3 writes u
and reads w2 around it and u at the item, each node of u read and then
overwritten by the same thread). It also checks that the schedule never
stalls, whatever the number of blocks."""
import heapq

import numpy as np
import pytest


def simulate(nrb, nseg, steps, blocks, seed, wait_reach=1):
    rng = np.random.default_rng(seed)
    items = nrb * nseg
    epochs = 3 * steps
    total = items * epochs
    done_at = {}                                 # (epoch, item) -> finish time
    # per (buffer, item): list of (epoch_written, start, finish) writes and the
    # reads of each version (start, finish, epoch of the version read)
    writes = {}
    reads = []

    def nbrs(item):
        rb, sg = divmod(item, nseg)
        for dr in (-1, 0, 1):
            for ds in (-1, 0, 1):
                r, g = rb + dr, sg + ds
                if 0 <= r < nrb and 0 <= g < nseg:
                    yield r * nseg + g

    next_ticket = 0
    events = []                                   # (time, block)
    cur, nxt = {}, {}                             # block -> current, prefetched ticket

    def grab():
        nonlocal next_ticket
        t = next_ticket
        next_ticket += 1
        return t

    for b in range(blocks):
        cur[b], nxt[b] = grab(), None
        heapq.heappush(events, (0.0, b))
    finished = 0
    parked = []                                   # blocks waiting for an item to start
    while events or parked:
        if not events:
            raise AssertionError("schedule deadlocked: every block waits")
        now, b = heapq.heappop(events)
        t = cur[b]
        if t >= total:
            continue
        if nxt[b] is None:
            nxt[b] = grab()                       # taken as soon as the block reads t
        e, item = divmod(t, items)
        # the earliest start: every neighbour has finished epoch e - 1
        start = now
        if e > 0:
            deps = nbrs(item) if wait_reach else [item]
            need = [done_at.get((e - 1, n)) for n in deps]
            if any(x is None for x in need):
                # a neighbour has not started epoch e - 1: wait for a start
                parked.append((now, b))
                continue
            start = max([now] + need)
        dur = rng.uniform(0.5, 1.5)
        fin = start + dur
        stage = e % 3 + 1
        step = e // 3
        # buffers read: (buffer, items, version epoch expected)
        prev_u = 3 * step - 1                     # stage 3 of the previous step (-1: initial)
        if stage == 1:
            rd = [("u", list(nbrs(item)), prev_u)]
            wr = "w1"
        elif stage == 2:
            rd = [("w1", list(nbrs(item)), e - 1), ("u", [item], prev_u)]
            wr = "w2"
        else:
            rd = [("w2", list(nbrs(item)), e - 1), ("u", [item], prev_u)]
            wr = "u"
        for buf, its, ver in rd:
            for j in its:
                reads.append((buf, j, ver, start, fin, e))
        writes.setdefault((wr, item), []).append((e, start, fin))
        done_at[(e, item)] = fin
        finished += 1
        cur[b], nxt[b] = nxt[b], None
        heapq.heappush(events, (fin, b))
        for tw, bw in parked:                     # an item started: retry the waiters
            heapq.heappush(events, (max(tw, start), bw))
        parked = []
    assert finished == total
    # check every read against the writes of its buffer and item
    for buf, j, ver, s, f, e_r in reads:
        ws = sorted(writes.get((buf, j), []))
        for e_w, sw, fw in ws:
            if e_w == ver:
                assert fw <= s, f"read of {buf}[{j}] (version {ver}) starts before it is written"
            elif e_w == e_r:
                # stage 3 reads u^n at each node and then overwrites that node
                # in the same thread: in place, not a race
                continue
            elif e_w > ver:
                # the next version may only be written after this read ended
                assert sw >= f, f"{buf}[{j}] overwritten (epoch {e_w}) while version {ver} is read"
                break
        if ver >= 0:
            assert any(e_w == ver for e_w, _, _ in ws), (buf, j, ver)


@pytest.mark.parametrize("nrb,nseg,steps,blocks", [
    (1, 1, 4, 1), (1, 5, 3, 2), (3, 1, 3, 7), (4, 4, 3, 5), (6, 9, 4, 16),
    (8, 8, 2, 200), (5, 7, 5, 3), (32, 64, 2, 1216 // 8)])
def test_fused_schedule_orders_every_read_and_write(nrb, nseg, steps, blocks):
    for seed in range(3):
        simulate(nrb, nseg, steps, blocks, seed)


def test_the_model_detects_a_missing_neighbour_wait():
    """With a wait on the item itself only, some stencil read overlaps a
    write: the check above has teeth."""
    with pytest.raises(AssertionError):
        for seed in range(20):
            simulate(2, 3, 3, 6, seed, wait_reach=0)


def simulate_withheld(nrb, nseg, steps, blocks, seed, wait_bound=4.0):
    """The same schedule with item 0's first completion never published (the
    kernel's test hook) and the kernel's wait rules: a block takes its ticket,
    reads the neighbours' flags, and if one is not yet set spins until it is,
    until another block has raised the abort word (then it stops), or until
    its own wait has lasted wait_bound (then it raises abort and stops); a
    block whose neighbourhood is ready computes whatever the abort word says.
    Returns (items completed, blocks that stopped on abort, abort raised)."""
    rng = np.random.default_rng(seed)
    items = nrb * nseg
    total = items * 3 * steps
    done_at = {}

    def nbrs(item):
        rb, sg = divmod(item, nseg)
        for dr in (-1, 0, 1):
            for ds in (-1, 0, 1):
                r, g = rb + dr, sg + ds
                if 0 <= r < nrb and 0 <= g < nseg:
                    yield r * nseg + g

    next_ticket = blocks
    events = [(0.0, b, b, None) for b in range(blocks)]    # (time, block, ticket, spin start)
    heapq.heapify(events)
    abort = None
    completed = stopped = 0
    guard = 0
    while events:
        guard += 1
        assert guard < 100 * total + 10 * blocks, "schedule did not end"
        now, b, t, spin0 = heapq.heappop(events)
        if t >= total:
            continue
        e, item = divmod(t, items)
        need = [] if e == 0 else [done_at.get((e - 1, n)) for n in nbrs(item)]
        if any(x is None or x > now for x in need):
            if spin0 is None:
                spin0 = now
            if abort is not None and abort <= now:
                stopped += 1
                continue
            if now >= spin0 + wait_bound:
                abort = now if abort is None else abort
                stopped += 1
                continue
            known = [x for x in need if x is not None and x > now]
            wake = min(known + [spin0 + wait_bound, now + 0.25])
            heapq.heappush(events, (wake, b, t, spin0))
            continue
        fin = now + rng.uniform(0.5, 1.5)
        if not (e == 0 and item == 0):                     # the withheld flag
            done_at[(e, item)] = fin
        completed += 1
        heapq.heappush(events, (fin, b, next_ticket, None))
        next_ticket += 1
    return completed, stopped, abort is not None


@pytest.mark.parametrize("nrb,nseg,steps,blocks", [(4, 4, 3, 5), (6, 9, 4, 16), (8, 8, 2, 200)])
def test_a_withheld_flag_ends_the_launch(nrb, nseg, steps, blocks):
    """Every block ends: the waits that depend on the withheld flag run out,
    raise abort, and every block that then has to wait stops, while work whose
    neighbourhood is ready may still finish; the launch ends early."""
    for seed in range(3):
        completed, stopped, aborted = simulate_withheld(nrb, nseg, steps, blocks, seed)
        assert aborted
        assert 0 < completed < nrb * nseg * 3 * steps
        assert stopped >= 1
