"""Host-side logic of bench.py that needs no GPU: the algorithmic byte count, and the
multi-rank reduction (max over ranks, barrier) on gloo with world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_bytes_per_lu():
    # populations 9 (N + 2) and lagged planes 3 + 2 N, read + written once, 8 bytes
    assert bench.bytes_per_lu(2) == 688
    assert bench.bytes_per_lu(3) == 864
    assert bench.bytes_per_lu(4) == 1040
    assert bench.bytes_per_lu(2, "fp32") == 344
    assert bench.bytes_per_lu(2, "fp16s") == 216


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    v = bench.reduce_max(1.5 + rank, world)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, v))


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 2.5, 1: 2.5}
