"""The multi-GPU path of the benchmark on CPU ranks (gloo, world size 2).

Chains shard by rank with no data-path collective: each rank owns chains with
distinct Philox chain ids, and the only exchange is the final (max time, sum of
accepted updates) reduction.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    chains, _ = bench.workload("cube8", 256.0, 64, chain_id=rank)
    ms = 100.0 + 10.0 * rank           # rank 1 is the slow one
    acc = 1000 + rank
    total_ms, acc_sum = bench.reduce_over_ranks(torch, dist, ms, acc, "cpu")
    q.put((rank, chains[0].chain_id, chains[0].seed, total_ms, acc_sum))
    dist.destroy_process_group()


def test_two_ranks_shard_chains_and_reduce_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, id0, s0, t0, a0), (r1, id1, s1, t1, a1) = res
    assert id0 != id1 and s0 != s1               # independent Philox streams per rank
    assert t0 == t1 == 110.0                     # the slowest rank's time
    assert a0 == a1 == 2001.0                    # accepted updates of the whole job
