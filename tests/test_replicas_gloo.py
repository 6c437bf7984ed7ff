"""The N > 1 (replica) bookkeeping under torch.distributed with the gloo
backend on CPU, world size 2: max-over-ranks timing, the whole-job rate, and
the flop-balanced sharding of a ragged batch (every matrix on exactly one
rank)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0709_1272_gb300 import inputs, replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + rank * 0.5
        t = replicas.max_over_ranks(t_local, dist)
        shapes = inputs.batch_shapes(101, seed=42)
        costs = [2.0 * n * n * (m - n / 3.0) for m, n in shapes]
        parts = replicas.shard_batch(costs, world)
        mine = sum(costs[b] for b in parts[rank])
        tot = replicas.job_rate([sum(costs[b] for b in p) for p in parts], t)
        results[rank] = (t, parts, mine, tot)
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_bookkeeping():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), results), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(results)
    assert set(res) == {0, 1}
    t0, parts0, mine0, rate0 = res[0]
    t1, parts1, mine1, rate1 = res[1]
    assert t0 == t1 == 1.5                       # the slower rank's time on every rank
    assert parts0 == parts1                      # every rank computes the same split
    allidx = sorted(parts0[0] + parts0[1])
    assert allidx == list(range(101))            # each matrix exactly once
    assert abs(mine0 - mine1) / max(mine0, mine1) < 0.02   # flop-balanced
    assert rate0 == pytest.approx((mine0 + mine1) / 1.5)


def test_single_process_defaults():
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.shard_batch([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
