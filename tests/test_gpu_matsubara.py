"""Measurement in Matsubara frequencies on the GPU against the oracle (needs a GB300).

Per configuration, G_xy(i w_n) of the CUDA path (S_zw by site pairs, exact
transform of the interpolated G0 table) against oracle.measure_G_matsubara
(einsum over the explicit M = (e^V - 1) N, Simpson transform of the table):
FP64 within 1e-9 of max|G|, the mixed form within 1e-4 of max|G|.
"""
import numpy as np
import pytest

from parity import compare_config, oracle_for
from oracle.ctaux import cluster_momenta
from workloads import configs

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1010_3690_gb300")


def _quadrature_tol(ch, n_freq):
    """The oracle transforms the table by Simpson's rule per interval, which
    leaves a relative error of order (w dtau)^4 / 2880 against the exact
    integral the GPU evaluates; allow 10x that, and at least 1e-9."""
    wdt = (2 * n_freq - 1) * np.pi / ch.beta * ch.beta / (ch.n_tau - 1)
    return max(1e-9, wdt ** 4 / 288.0)


def _one_measurement(ch, n0, n_freq, prec, seed=5):
    cfg = configs.synthetic_configuration(ch, n0, seed=seed) if n0 else None
    oc = oracle_for(ch)
    with pk.Context([ch], precision=prec, n_matsubara=n_freq) as ctx:
        if cfg is not None:
            oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
            ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.reset_measurements()
        ctx.sweep(1, measure=True)
        G, E, nm = ctx.measure_G_matsubara(0)
        assert nm == 1
        oc.run(ctx.stats(0)["t"] - oc.t)   # a near tie can end the block early
        compare_config(ctx, 0, oc)
    return G, oc.measure_G_matsubara(n_freq), oc


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("maker,n0,n_freq", [("cube8", 60, 8), ("cube8", 430, 16),
                                             ("aim1", 0, 64), ("cube8", 200, 3)])
def test_matsubara_measurement_matches_oracle(maker, n0, n_freq, prec):
    ch = (configs.cube8(K=256.0, k_max=32, capacity=768) if maker == "cube8"
          else configs.aim1(K=1.0, k_max=8, capacity=128))
    G, ref, oc = _one_measurement(ch, n0, n_freq, prec)
    assert G.shape == ref.shape == (2, ch.n_c, ch.n_c, n_freq)
    scale = np.abs(ref).max()
    err = np.abs(G - ref).max() / scale
    print(f"{maker} n={oc.order} F={n_freq} precision {prec}: max |G - G_oracle| / max|G| = {err:.2e}")
    assert err <= (_quadrature_tol(ch, n_freq) if prec == 0 else 1e-4), err


def test_matsubara_empty_configuration_is_g0_and_momenta():
    """n = 0: G = G0(i w), the table's transform; its cluster-momentum transform is
    diagonal in K and equal for both spins (paramagnetic table)."""
    ch = configs.cube8(K=1.0, k_max=8, capacity=64)
    oc = oracle_for(ch)
    with pk.Context([ch], n_matsubara=12, p_insert=0.0) as ctx:   # removals only: stays empty
        ctx.reset_measurements()
        ctx.sweep(2, measure=True)
        G, E, nm = ctx.measure_G_matsubara(0)
        assert nm == 2 and ctx.stats(0)["n"] == 0
    ref = oc.measure_G_matsubara(12)
    np.testing.assert_allclose(G, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    cl = configs.cluster(8)
    GK = cluster_momenta(G, cl.sites, cl.K)
    np.testing.assert_allclose(GK[0], GK[1], rtol=0, atol=1e-14)
    # two identical measurements: the naive error is cancellation noise
    assert np.abs(E).max() <= 1e-7 * np.abs(ref).max()


def test_matsubara_batched_chains_and_accumulation():
    """Chains of different cluster sizes in one context: each chain's accumulated
    mean over three measurements equals the mean of the oracle's estimates."""
    chs = [configs.cube8(K=64.0, k_max=16, capacity=512, seed=3)]
    pool = configs.batch(n_chains=30, k_max=16, n_tau=512)
    chs += [next(c for c in pool if c.n_c == 4), next(c for c in pool if c.n_c == 16)]
    for i, c in enumerate(chs):
        c.chain_id = 100 + i
    F = 6
    with pk.Context(chs, n_matsubara=F, trace_capacity=256) as ctx:
        ctx.sweep(8)
        ctx.reset_measurements()
        ctx.sweep(3, measure=True)
        got = [ctx.measure_G_matsubara(i) for i in range(len(chs))]
    for i, ch in enumerate(chs):
        oc = oracle_for(ch)
        oc.run(8 * ch.k_max)
        acc = []
        for _ in range(3):
            oc.run(ch.k_max)
            acc.append(oc.measure_G_matsubara(F))
        ref = np.mean(acc, axis=0)
        G, E, nm = got[i]
        assert nm == 3
        tol = _quadrature_tol(ch, F)
        err = np.abs(G - ref).max() / np.abs(ref).max()
        print(f"batched N_c={ch.n_c} n_tau={ch.n_tau}: {err:.2e} (tolerance {tol:.1e})")
        assert err <= tol, err
