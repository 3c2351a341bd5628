"""History-id sharding over ranks (the multi-GPU path) on CPU, through the
product's sharding code (paper_2304_06226_gb300.shard): two gloo ranks each
take their share of the history ids (shard_range), run them -- the oracle
stands in for the device tallies, since this machine has no GPU -- and combine
sum w, sum w^2, the score-function tallies and the history counts with the one
FP64 all-reduce of reduce_sums.  The result equals one process running every
id, because the random numbers are keyed by history id and not by rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2304_06226_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, grad, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.oracle import OracleScene
    desc = W.batched(n_instances=2, seed=7) if grad else W.slab(g=3.0, n_histories=n)
    first, cnt = shard.shard_range(n, rank, world)
    r = OracleScene(desc).run(cnt, first=first, threads=2, want_grad=grad)
    parts = {"sum": torch.tensor(r["sum"]), "sumsq": torch.tensor(r["sumsq"]),
             "n": torch.tensor([float(cnt)], dtype=torch.float64)}
    if grad:
        parts["J"] = torch.tensor(r["J"])
        parts["J2"] = torch.tensor(r["J2"])
    shard.reduce_sums(parts)
    if rank == 0:
        out.put({k: v.numpy() for k, v in parts.items()})
    dist.destroy_process_group()


def _spawn(n, grad):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, n, grad, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


@pytest.mark.parametrize("grad", [False, True])
def test_two_ranks_add_up_to_one_run(grad):
    n = 60_001 if not grad else 20_001       # odd: the shares differ by one history
    got = _spawn(n, grad)
    from oracle.oracle import OracleScene
    desc = W.batched(n_instances=2, seed=7) if grad else W.slab(g=3.0, n_histories=n)
    full = OracleScene(desc).run(n, threads=4, want_grad=grad)
    assert got["n"][0] == n
    for k in ("sum", "sumsq") + (("J", "J2") if grad else ()):
        assert np.allclose(got[k], full[k], rtol=1e-12, atol=1e-14), k


def test_shard_ranges_partition_the_ids():
    for n in (0, 1, 7, 1000, 10**9 + 3):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0
            for (f0, c0), (f1, _) in zip(spans, spans[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in spans) == n
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


@pytest.mark.parametrize("world,n", [(4, 1000), (8, 1_000_000_000)])
def test_step_streams_never_repeat_a_history(world, n):
    seen = set()
    for step in range(5):
        for r in range(world):
            key, first = shard.step_stream(step, r, world, n, seed=4096)
            assert first + n <= 2 ** 32
            span = (key, first, first + n)
            for k2, a, b in seen:
                assert k2 != key or b <= first or first + n <= a, (span, (k2, a, b))
            seen.add(span)


def test_reduce_sums_rejects_reduced_precision():
    t = {"sum": torch.zeros(3, dtype=torch.float32)}
    with pytest.raises(TypeError):
        shard.reduce_sums(t)
