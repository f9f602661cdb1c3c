"""Host-side logic of the y-slab decomposition that needs no GPU: the band split, the
neighbours, the order of the halo exchange and the all-reduce of the diagnostics sums,
on gloo with world size 2 (the GPU path runs the same schedule over NCCL, with the
packing done by the library's kernels).

The bands here are stand-ins that carry tagged rows instead of populations: a step
writes, per band, the rows it pushed across each cut (ghost rows) and its own boundary
rows; after the exchange, (phase 1) each boundary row must hold what the neighbour pushed
across the cut, and (phase 2) each ghost row must hold the neighbour's boundary row as
phase 1 left it, both for an open and for a periodic lattice, in which the two ranks are
each other's upper and lower neighbour."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2603_22902_gb300 import slab as S

W = 5  # values per row


def tag(rank, kind, step):
    return np.full(W, 1000.0 * rank + 100.0 * kind + step)


PUSH_UP, PUSH_DOWN, FIRST, LAST = 1, 2, 3, 4


class FakeBand:
    """Rows of a band: ghost below / above, first / last own row."""

    def __init__(self, rank):
        self.rank = rank
        self.n = 0
        self.log = []
        self.rows = {k: np.zeros(W) for k in ("ghost_below", "first", "last", "ghost_above")}
        self.msg_bytes = {1: 8 * W, 2: 8 * W}

    def step(self, n):
        self.n += n
        r = self.rows
        r["ghost_above"][:] = tag(self.rank, PUSH_UP, self.n)
        r["ghost_below"][:] = tag(self.rank, PUSH_DOWN, self.n)
        r["first"][:] = tag(self.rank, FIRST, self.n)
        r["last"][:] = tag(self.rank, LAST, self.n)

    def step_part(self, part):
        # the inner part touches none of the rows here; the edge part completes the step
        self.log.append(("inner" if part == S.INNER else "edge", self.n + 1))
        if part == S.EDGE:
            self.step(1)

    def pack(self, side, phase, msg):
        if phase == 1:
            src = "ghost_above" if side == S.YMAX else "ghost_below"
        else:
            src = "last" if side == S.YMAX else "first"
        msg.copy_(torch.from_numpy(self.rows[src]))

    def unpack(self, side, phase, msg):
        if phase == 1:
            dst = "first" if side == S.YMIN else "last"
        else:
            dst = "ghost_below" if side == S.YMIN else "ghost_above"
        self.rows[dst][:] = msg.numpy()

    def sums(self):
        r = self.rank
        return dict(mass=[1.0 + r, 2.0 + r], solid=[0.5 * r, 0.25], max_sum_dev=1e-14 * (r + 1), nonfinite=r)


def test_split_and_neighbours():
    assert S.split_rows(10, 3) == [(0, 3), (3, 7), (7, 10)]
    assert S.split_rows(512, 2) == [(0, 256), (256, 512)]
    with pytest.raises(ValueError):
        S.split_rows(4, 5)
    assert S.neighbours(0, 3, False) == (None, 1)
    assert S.neighbours(2, 3, False) == (1, None)
    assert S.neighbours(0, 3, True) == (2, 1)
    assert S.neighbours(0, 2, True) == (1, 1)
    assert S.neighbours(0, 1, True) == (None, None)


def test_combine_sums():
    a = dict(mass=[1.0, 2.0], solid=[0.0, 0.5], max_sum_dev=3e-15, nonfinite=0)
    b = dict(mass=[0.5, 4.0], solid=[1.0, 0.0], max_sum_dev=7e-15, nonfinite=2)
    c = S.combine_sums([a, b], 2)
    assert c == dict(mass=[1.5, 6.0], solid=[1.0, 0.5], max_sum_dev=7e-15, nonfinite=2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, periodic, q, overlap=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    band = FakeBand(rank)
    ex = S.DistExchange(band, periodic, alloc=lambda n: torch.zeros(n // 8, dtype=torch.float64))
    plain_exchange = ex.exchange

    def logged_exchange():
        band.log.append(("exchange", band.n))
        plain_exchange()

    ex.exchange = logged_exchange
    out = []
    if overlap:
        ex.step(3, overlap=True)
        out = [None, None, {k: v.copy() for k, v in band.rows.items()}]
    else:
        for _ in range(3):
            ex.step(1)
            out.append({k: v.copy() for k, v in band.rows.items()})
    out.append(band.log)
    sums = ex.sums(2)
    dist.destroy_process_group()
    q.put((rank, out, sums))


@pytest.mark.parametrize("periodic", [False, True])
def test_exchange_order_and_sums_on_two_gloo_ranks(periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, periodic, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, out, sums = q.get(timeout=120)
        res[r] = (out, sums)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    check_rows(res, periodic, range(3))


def check_rows(res, periodic, which):
    for n in which:
        step = n + 1
        lo, hi = res[0][0][n], res[1][0][n]
        # phase 1: the rows pushed across the 0|1 cut arrive in the boundary rows
        assert np.array_equal(hi["first"], tag(0, PUSH_UP, step))
        assert np.array_equal(lo["last"], tag(1, PUSH_DOWN, step))
        # phase 2: the ghost rows hold the neighbour's boundary row after phase 1
        assert np.array_equal(hi["ghost_below"], tag(1, PUSH_DOWN, step))
        assert np.array_equal(lo["ghost_above"], tag(0, PUSH_UP, step))
        if periodic:
            # the 1|0 cut through the periodic side, the other way round
            assert np.array_equal(lo["first"], tag(1, PUSH_UP, step))
            assert np.array_equal(hi["last"], tag(0, PUSH_DOWN, step))
            assert np.array_equal(lo["ghost_below"], tag(0, PUSH_DOWN, step))
            assert np.array_equal(hi["ghost_above"], tag(1, PUSH_UP, step))
        else:
            # no cut beyond the global sides: those rows keep what the step wrote
            assert np.array_equal(lo["first"], tag(0, FIRST, step))
            assert np.array_equal(hi["last"], tag(1, LAST, step))
    expect = S.combine_sums([FakeBand(0).sums(), FakeBand(1).sums()], 2)
    for r in (0, 1):
        got = res[r][1]
        assert got["mass"] == expect["mass"] and got["solid"] == expect["solid"]
        assert got["max_sum_dev"] == expect["max_sum_dev"] and got["nonfinite"] == expect["nonfinite"]


@pytest.mark.parametrize("periodic", [False, True])
def test_overlapped_schedule_on_two_gloo_ranks(periodic):
    # step(3, overlap=True): per step the inner part, the previous step's exchange, the edge
    # part; the last exchange after the loop.  The rows end as after three plain steps.
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, periodic, q, True)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, out, sums = q.get(timeout=120)
        res[r] = (out, sums)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    check_rows(res, periodic, [2])
    for r in (0, 1):
        log = res[r][0][3]
        assert log == [("inner", 1), ("edge", 1), ("inner", 2), ("exchange", 1), ("edge", 2),
                       ("inner", 3), ("exchange", 2), ("edge", 3), ("exchange", 3)], log
