"""The multi-GPU path of the benchmark on CPU ranks (gloo, world size 2).

Chains shard by rank with no data-path collective: each rank owns chains with
distinct Philox chain ids.  The exchanges are the final (max time, sum of
accepted updates) reduction and the all-reduce of the G(tau) measurement
accumulators (sums, squares, bin sums and counts).  Here each rank builds real
accumulators from oracle measurements of its own chains, and the all-reduced
estimate must equal the one a single process computes from every measurement.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BINS, ANCHORS, BIN_SIZE, N_MEAS, K_BLOCK = 6, 2, 4, 24, 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_measurements(chain_id):
    """Per-configuration G estimates of one oracle chain (one after every block)."""
    sys.path.insert(0, ROOT)
    from oracle.ctaux import OracleChain
    from workloads import configs
    ch = configs.aim1(K=1.0, k_max=K_BLOCK, capacity=128, seed=chain_id)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=chain_id, chain_id=chain_id)
    oc.run(200)
    out = []
    for _ in range(N_MEAS):
        oc.run(K_BLOCK)
        out.append(oc.measure_G(BINS, ANCHORS))
    return np.array(out)


def _accumulate(meas):
    """The accumulators of ctaux_get_accumulators, built from a list of estimates."""
    bm = meas.reshape(-1, BIN_SIZE, *meas.shape[1:]).mean(axis=1)
    return dict(sum=meas.sum(axis=0), sumsq=(meas ** 2).sum(axis=0), bin_sum=bm.sum(axis=0),
                bin_sumsq=(bm ** 2).sum(axis=0), n_meas=len(meas), n_bins=len(bm),
                bin_size=BIN_SIZE)


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
    # two chains per rank, distinct ids across ranks
    accs = [_accumulate(_oracle_measurements(2 * rank + j)) for j in range(2)]
    mean, err, n_meas, n_bins = bench.merge_accumulators(torch, dist, bench.pool_accumulators(accs),
                                                         "cpu")
    q.put((rank, chains[0].chain_id, chains[0].seed, total_ms, acc_sum, mean, err, n_meas, n_bins))
    dist.destroy_process_group()


def test_two_ranks_shard_chains_and_merge_measurements():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r0, r1 = res
    assert r0[1] != r1[1] and r0[2] != r1[2]          # independent Philox streams per rank
    assert r0[3] == r1[3] == 110.0                    # the slowest rank's time
    assert r0[4] == r1[4] == 2001.0                   # accepted updates of the whole job
    # the merged estimate: identical on both ranks and equal to one process pooling
    # all four chains' measurements
    allm = np.concatenate([_oracle_measurements(c) for c in range(4)])
    bm = np.concatenate([_oracle_measurements(c).reshape(-1, BIN_SIZE, *allm.shape[1:]).mean(axis=1)
                         for c in range(4)])
    want_mean = allm.mean(axis=0)
    want_err = bm.std(axis=0, ddof=1) / np.sqrt(len(bm))
    for r in res:
        mean, err, n_meas, n_bins = r[5:]
        assert n_meas == 4 * N_MEAS and n_bins == 4 * N_MEAS // BIN_SIZE
        np.testing.assert_allclose(mean, want_mean, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(err, want_err, rtol=1e-8, atol=1e-14)
    assert np.all(np.isfinite(res[0][6])) and np.any(res[0][6] > 0)


def test_pooled_estimate_single_process():
    """pool_accumulators + pooled_estimate on one host: the same numbers as
    pooling the raw measurements (no collective)."""
    sys.path.insert(0, ROOT)
    import bench
    meas = [_oracle_measurements(c) for c in (7, 8)]
    acc = bench.pool_accumulators([_accumulate(m) for m in meas])
    mean, err, n_meas, n_bins = bench.pooled_estimate(acc["sum"], acc["bin_sum"], acc["bin_sumsq"],
                                                      acc["n_meas"], acc["n_bins"])
    allm = np.concatenate(meas)
    np.testing.assert_allclose(mean, allm.mean(axis=0), rtol=1e-12, atol=1e-14)
    assert n_meas == 2 * N_MEAS
    with pytest.raises(AssertionError):      # a planted wrong count is seen
        np.testing.assert_allclose(acc["sum"] / (n_meas - 1), allm.mean(axis=0), rtol=1e-6)
