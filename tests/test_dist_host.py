"""The multi-rank host logic of bench.py (one process per GPU, replicas with no data-path
collective) on CPU: two gloo ranks on 127.0.0.1 synchronise with the bench's barrier, agree
on the maximum of their step times, and draw distinct right-hand-side batches."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import inputs
        bench.barrier(world)
        t = bench.max_over_ranks(1.5 + rank, world, device="cpu")
        c, p = inputs.bump_batch(bench.rhs_seed(rank), 2)
        out[rank] = (t, float(c.sum()), float(np.abs(p).sum()))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(120)
            assert pr.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5  # both ranks see the slowest time
    assert res[0][1] != res[1][1]  # distinct right-hand-side batches per rank

