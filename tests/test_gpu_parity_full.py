"""CUDA path against the oracle at the benchmark's full sizes (needs a GB300).

The workloads the benchmark times reach orders the oracle (a dense LU per
proposal) cannot replay for long, so each case starts both sides from the
same seeded configuration and compares:
  * the proposals the oracle replays one by one (a prefix of a block, or whole
    blocks where that takes seconds): same counter, move, vertex, proposed spin
    and accept decision, determinant ratios within the form's tolerance;
  * N after the block against the property that holds at any size:
    N = (N^{-1})^{-1} of the configuration the chain ends in, with N^{-1} built
    by the oracle (Eq. Nmatrix) and inverted by numpy.
Ratio errors of the mixed form are printed with each case.
"""
import numpy as np
import pytest

from parity import compare_config, compare_traces, oracle_for
from workloads import configs

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1010_3690_gb300")

RTOL64 = 1e-10
RTOL_MIXED = 1e-5


def _start(ctx, chains, order, seed0=1000):
    cfgs = []
    for i, ch in enumerate(chains):
        cfg = configs.synthetic_configuration(ch, order, seed=seed0 + ch.chain_id)
        ctx.set_config(i, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        cfgs.append(cfg)
    return cfgs


def _check_N_is_inverse(ctx, chain, oc_like, rtol):
    """Property check at any size: the chain's N against the inverse of N^{-1}
    built (Eq. Nmatrix) from the configuration the chain ends in."""
    cfg = ctx.get_config(chain)
    worst = 0.0
    for spin in (0, 1):
        A = oc_like.ninv(spin, cfg["tau"], cfg["site"].astype(np.int64), cfg["s"].astype(np.int64))
        ref = np.linalg.inv(A)
        got = ctx.get_N(chain, spin)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        assert err <= rtol, (spin, err)
    return worst


def _forms():
    return [("fp64", pk.CTAUX_FP64, RTOL64, 1e-8), ("mixed", pk.CTAUX_MIXED, RTOL_MIXED, 1e-4)]


@pytest.mark.parametrize("gamma", ["inverse", "lu"])
def test_cube100_full_size_k256_prefix_and_flush(gamma):
    """The 100-site cluster as the benchmark runs it: K=5700, k_max=256, 8 chains
    started at order 7000, one block, Gamma as its inverse or as L U.  Chain 0's
    first proposals against the oracle (about a second each at this order), and
    every chain's N after the rank-k_acc flush (k_acc ~ 220) against the inverse
    of its configuration."""
    n_chains, order, n_replay = 8, 7000, 10
    chains = [configs.cube100(K=5700.0, k_max=256, capacity=9216, seed=i, chain_id=i)
              for i in range(n_chains)]
    oc = oracle_for(chains[0])
    cfg0 = configs.synthetic_configuration(chains[0], order, seed=1000)
    oc.set_config(cfg0["tau"], cfg0["site"], cfg0["s"], cfg0["birth"], cfg0["t"])
    recs = oc.run(n_replay)
    for name, prec, rtol, ntol in _forms():
        with pk.Context(chains, precision=prec, trace_capacity=256, refresh_every=0,
                        use_graph=1, gamma_form=1 if gamma == "lu" else 0) as ctx:
            _start(ctx, chains, order)
            ctx.sweep(1, measure=True)
            ctx.synchronize()
            tr = ctx.trace(0)
            # the mixed form ends a block early at a near tie (decided in FP64)
            assert len(tr) == 256 if prec == pk.CTAUX_FP64 else 0 < len(tr) <= 256
            k = min(n_replay, len(tr))
            worst = compare_traces(tr[:k], recs[:k], rtol)
            st = ctx.stats(0)
            k_acc = int(sum(st["accepted"]))
            errs = [_check_N_is_inverse(ctx, c, oc, ntol) for c in (0, n_chains - 1)]
            print(f"cube100 {name} {gamma}: worst ratio error {worst:.2e} over {k} proposals, "
                  f"{k_acc} accepted in the block, N error {max(errs):.2e}")


@pytest.mark.parametrize("name,prec,rtol", [("fp64", 0, RTOL64), ("mixed", 1, RTOL_MIXED)])
def test_sq36_full_size_block_parity(name, prec, rtol):
    """The 6x6 cluster at density 0.9 (sign can be negative), K=1400, k_max=128,
    from a seeded configuration of order 2000: one whole block against the
    oracle, then N against the inverse of the final configuration."""
    ch = configs.sq36(K=1400.0, k_max=128, capacity=3072)
    cfg = configs.synthetic_configuration(ch, 2000, seed=21)
    oc = oracle_for(ch)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    with pk.Context([ch], precision=prec, trace_capacity=256, refresh_every=0) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.sweep(1)
        ctx.synchronize()
        tr = ctx.trace(0)
        recs = oc.run(len(tr))
        worst = compare_traces(tr, recs, rtol)
        compare_config(ctx, 0, oc)
        nerr = 0.0
        for spin in (0, 1):
            No = oc.N(spin)
            nerr = max(nerr, np.abs(ctx.get_N(0, spin) - No).max() / np.abs(No).max())
        assert nerr <= (1e-8 if prec == 0 else 1e-4), nerr
        st = ctx.stats(0)
        print(f"sq36 {name}: {len(tr)} proposals, worst ratio error {worst:.2e}, "
              f"near ties {st['near_ties']}, N error {nerr:.2e}, sign {st['sign']}")


@pytest.mark.parametrize("gamma", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_k256_whole_blocks_against_oracle(prec, gamma):
    """k_max = 256 (Gamma^{-1}, or L U, of 2 x 256 x 257 entries, kept in global
    memory) over three blocks of the 2x2x2 cluster at order 430.  In the mixed
    form a block ends early at a near tie (decided in FP64 and applied by the
    next block), so its trace holds at most 3 x 256 records."""
    ch = configs.cube8(K=256.0, k_max=256, capacity=1024)
    cfg = configs.synthetic_configuration(ch, 430, seed=5)
    oc = oracle_for(ch)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    with pk.Context([ch], precision=prec, trace_capacity=768, refresh_every=0,
                    gamma_form=gamma) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.sweep(3)
        ctx.synchronize()
        tr = ctx.trace(0)
        st = ctx.stats(0)
        assert len(tr) == 768 if prec == 0 else 256 < len(tr) <= 768
        worst = compare_traces(tr, oc.run(len(tr)), RTOL64 if prec == 0 else RTOL_MIXED)
        assert st["t"] == oc.t
        compare_config(ctx, 0, oc)
        print(f"cube8 k=256 precision {prec} gamma {gamma}: {len(tr)} proposals, "
              f"worst ratio error {worst:.2e}, "
              f"near ties {st['near_ties']}")


def test_batch_chains_of_every_cluster_size_against_oracle():
    """Chains of the batch workload with N_c = 4, 8 and 16 (uneven beta, U, K),
    run together in one context, each against its own oracle replay."""
    pool = configs.batch(n_chains=40, k_max=16, n_tau=512)
    picked = []
    for nc in (4, 8, 16):
        picked += [c for c in pool if c.n_c == nc][:2]
    assert sorted({c.n_c for c in picked}) == [4, 8, 16]
    n_sw = 12
    with pk.Context(picked, trace_capacity=n_sw * 16, refresh_every=5) as ctx:
        ctx.sweep(n_sw)
        ctx.synchronize()
        for i, ch in enumerate(picked):
            tr = ctx.trace(i)
            oc = oracle_for(ch)
            compare_traces(tr, oc.run(len(tr)), RTOL64)
            compare_config(ctx, i, oc)


@pytest.mark.parametrize("prec", [0, 1])
def test_refresh_on_every_resident_cta_grid(prec):
    """A context whose refresh at capacity has more than 4096 trailing-update
    tiles per panel refreshes on the grid of every resident CTA (not one CTA per
    SM): its N against the oracle's, then two blocks of proposals."""
    ch = configs.cube8(K=256.0, k_max=64, capacity=1600)
    tb = (ch.capacity + ch.k_max + 31) // 32
    assert 2 * tb * tb > 4096
    cfg = configs.synthetic_configuration(ch, 430, seed=8)
    oc = oracle_for(ch)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    with pk.Context([ch], precision=prec, trace_capacity=256, refresh_every=1) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        tol = 1e-10 if prec == 0 else 1e-6
        for spin in (0, 1):
            No = oc.N(spin)
            np.testing.assert_allclose(ctx.get_N(0, spin), No, rtol=tol, atol=tol * np.abs(No).max())
        ctx.sweep(2)
        ctx.synchronize()
        tr = ctx.trace(0)
        compare_traces(tr, oc.run(len(tr)), RTOL64 if prec == 0 else RTOL_MIXED)
        compare_config(ctx, 0, oc)
        assert ctx.stats(0)["refreshes"] >= 3


@pytest.mark.parametrize("prec", [0, 1])
def test_measurement_above_1024_vertices(prec):
    """Orders above 1024 evaluate the estimator in 32-vertex chunks: the
    measurement of one configuration against the oracle's (C9)."""
    ch = configs.cube8(K=1024.0, k_max=32, capacity=1536)
    cfg = configs.synthetic_configuration(ch, 1100, seed=6)
    oc = oracle_for(ch)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    with pk.Context([ch], precision=prec, n_tau_bins=12, n_anchors=3) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.reset_measurements()
        ctx.sweep(1, measure=True)
        G, E, nm = ctx.measure_G(0)
        assert nm == 1
        oc.run(ctx.stats(0)["t"] - oc.t)   # a near tie can end the block early
        compare_config(ctx, 0, oc)
        assert oc.order > 1024
        ref = oc.measure_G(12, 3)
        if prec == 0:
            np.testing.assert_allclose(G, ref, rtol=1e-9, atol=1e-11)
        else:
            np.testing.assert_allclose(G, ref, rtol=0, atol=1e-4 * np.abs(ref).max())
