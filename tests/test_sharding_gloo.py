"""History-id sharding over ranks (the multi-GPU plan) on CPU: two gloo ranks
each run the oracle on their half of the history ids and sum their tallies
with an all-reduce; the result equals one process running every id, because
the random numbers are keyed by history id and not by rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.oracle import OracleScene
    desc = W.slab(g=3.0, n_histories=n)
    lo, hi = rank * n // world, (rank + 1) * n // world
    r = OracleScene(desc).run(hi - lo, first=lo, threads=2)
    t = torch.tensor(np.concatenate([r["sum"], r["sumsq"]]), dtype=torch.float64)
    dist.all_reduce(t)
    if rank == 0:
        out.put(t.numpy())
    dist.destroy_process_group()


def test_two_ranks_add_up_to_one_run():
    n = 60_000
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle.oracle import OracleScene
    full = OracleScene(W.slab(g=3.0, n_histories=n)).run(n, threads=4)
    tb = len(full["sum"])
    assert np.allclose(got[:tb], full["sum"], rtol=1e-12, atol=1e-12)
    assert np.allclose(got[tb:], full["sumsq"], rtol=1e-12, atol=1e-12)
