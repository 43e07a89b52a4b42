"""The CPU rank-one and submatrix algorithms of the benchmark's F2 comparison
(bench_cpu.py) run the oracle's Markov chain: same decisions, determinant
ratios within 1e-9, same configuration (no GPU needed)."""
import numpy as np
import pytest

import bench_cpu
from oracle.ctaux import OracleChain
from workloads import configs


def _setup(n0, K):
    ch = configs.cube8(K=K, k_max=32, capacity=1024)
    cfg = configs.synthetic_configuration(ch, n0, seed=4)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=ch.seed)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    model = bench_cpu.Model(ch.table, ch.dx_class, ch.beta, ch.U, ch.K)
    draws = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=ch.seed).draws
    return ch, cfg, oc, model, draws


def _compare(trace, recs, tau, s, Ns, oc):
    assert len(trace) == len(recs)
    for g, o in zip(trace, recs):
        assert g["t"] == o["t"] and g["move"] == o["move"] and g["n"] == o["n"]
        assert g["accept"] == o["accept"], (g, o)
        if o.get("birth", -1) >= 0:
            for sp in (0, 1):
                assert g["ratio"][sp] == pytest.approx(o["ratio"][sp], rel=1e-9, abs=1e-12)
    np.testing.assert_allclose(tau, oc.tau, rtol=0, atol=0)
    np.testing.assert_array_equal(s, oc.s)
    for spin in (0, 1):
        No = oc.N(spin)
        np.testing.assert_allclose(Ns[spin], No, rtol=1e-8, atol=1e-10 * np.abs(No).max())


@pytest.mark.parametrize("n0,K", [(0, 4.0), (120, 64.0)])
def test_rank_one_follows_the_oracle(n0, K):
    ch, cfg, oc, model, draws = _setup(n0, K)
    c = bench_cpu.RankOne(model, draws)
    c.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["t"])
    for _ in range(200):
        c.step()
    tau, site, s = c.config()
    _compare(c.trace, oc.run(200), tau, s, c.matrices(), oc)


@pytest.mark.parametrize("n0,K,k", [(0, 4.0, 8), (120, 64.0, 32), (60, 16.0, 64)])
def test_submatrix_follows_the_oracle(n0, K, k):
    ch, cfg, oc, model, draws = _setup(n0, K)
    c = bench_cpu.Submatrix(model, draws, k)
    c.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["t"])
    for _ in range(256 // k):
        c.block()
    _compare(c.trace, oc.run(len(c.trace)), c.tau, c.s, c.N, oc)
