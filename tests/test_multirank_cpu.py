"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards as independent replicas: each rank encodes its own copy,
the only exchange is the final max of times and sum of work across ranks,
and only rank 0 reports (the reference arm runs on rank 0 alone).
"""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import io
    import contextlib
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times, work = bench.rank_reduce([1.0 + rank, 5.0 - rank], [10 * (rank + 1), 7], "cpu")
    # the reference arm: only rank 0 does work and prints
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        if rank != 0:
            rc = bench.run_reference(type("A", (), dict(gpus=world, steps=1, warmup=0))())
        else:
            rc = 0
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, times, work, rc, buf.getvalue()))


def test_rank_reduce_and_reference_arm_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        rank, times, work, rc, printed = q.get(timeout=120)
        got[rank] = (times, work, rc, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        times, work, rc, _ = got[r]
        assert times == [2.0, 5.0]          # max over ranks
        assert work == [30.0, 14.0]         # sum over ranks
        assert rc == 0
    assert got[1][3] == ""                  # non-zero ranks print nothing
