"""Gamma kept as L U (Sec. III D, Eqs. lineq1-detrat) against the oracle and
against the partitioned inverse, through the C ABI (needs a GB300).

Both forms reach the same Markov chain: identical decisions and
configurations, ratios within the FP64 tolerance of the other parity tests.
The moves that make a slot change twice inside a block re-factorise L U by
Bennett's rank-one update; the traces are checked to contain both kinds (a
diagonal change of Gamma, and a slot returning to its block-start spin, which
deletes a row and column of the factors).
"""
import numpy as np
import pytest

from parity import compare_config, compare_traces, oracle_for
from workloads import configs

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1010_3690_gb300")

RTOL64 = 1e-10
RTOL_MIXED = 1e-5


def retouch_kinds(tr, k, n_blocks):
    """Accepted moves on a slot already changed earlier in the same block:
    (diagonal changes, returns to the block-start spin).  Blocks are k
    proposals long (FP64 form)."""
    diag = back = 0
    for b in range(n_blocks):
        start = {}
        for r in tr[b * k:(b + 1) * k]:
            if not (int(r["accept"]) & 1) or int(r["birth"]) < 0:
                continue
            v, s_new, mv = int(r["birth"]), int(r["s_new"]), int(r["move"])
            if v not in start:
                # spin before the first change: 0 for a pre-inserted vertex,
                # -s_new for a flip, some nonzero spin for a removal
                start[v] = 0 if mv == 0 else (-s_new if mv == 2 else None)
                continue
            if s_new == start[v]:
                back += 1
            else:
                diag += 1
    return diag, back


@pytest.mark.parametrize("K,k,n0,cap", [(4.0, 32, 0, 256), (256.0, 128, 430, 768)])
def test_lu_form_follows_the_oracle_with_retouches(K, k, n0, cap):
    """k = 32 keeps the factors in shared memory, k = 128 in global memory."""
    ch = configs.cube8(K=K, k_max=k, capacity=cap)
    n_blocks = 30 if n0 == 0 else 3
    oc = oracle_for(ch, p_insert=0.4, p_flip=0.3)
    with pk.Context([ch], trace_capacity=n_blocks * k, p_insert=0.4, p_flip=0.3,
                    refresh_every=8, gamma_form=pk.ctaux.CTAUX_GAMMA_LU) as ctx:
        if n0:
            cfg = configs.synthetic_configuration(ch, n0, seed=3)
            oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
            ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.sweep(n_blocks)
        ctx.synchronize()
        tr = ctx.trace(0)
        recs = oc.run(n_blocks * k)
        compare_traces(tr, recs, RTOL64)
        compare_config(ctx, 0, oc)
        for spin in (0, 1):
            No = oc.N(spin)
            np.testing.assert_allclose(ctx.get_N(0, spin), No, rtol=1e-8,
                                       atol=1e-10 * max(1.0, np.abs(No).max()))
    diag, back = retouch_kinds(tr, k, n_blocks)
    print(f"K={K} k={k}: accepted re-touches {diag} diagonal, {back} back to the start spin")
    assert diag > 0 and back > 0


def test_lu_and_inverse_forms_give_the_same_chain_at_k256():
    ch = configs.cube8(K=256.0, k_max=256, capacity=1024)
    cfg = configs.synthetic_configuration(ch, 500, seed=5)
    out = {}
    for form in (pk.ctaux.CTAUX_GAMMA_INVERSE, pk.ctaux.CTAUX_GAMMA_LU):
        with pk.Context([ch], trace_capacity=3 * 256, p_insert=0.4, p_flip=0.3,
                        refresh_every=0, gamma_form=form) as ctx:
            ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
            ctx.sweep(3)
            ctx.synchronize()
            out[form] = (ctx.trace(0), ctx.get_config(0), ctx.get_N(0, 0))
    a, b = out[pk.ctaux.CTAUX_GAMMA_INVERSE], out[pk.ctaux.CTAUX_GAMMA_LU]
    for f in ("t", "move", "n", "birth", "s_new", "accept"):
        np.testing.assert_array_equal(a[0][f], b[0][f])
    np.testing.assert_allclose(b[0]["ratio"], a[0]["ratio"], rtol=1e-10, atol=1e-10)
    np.testing.assert_array_equal(a[1]["birth"], b[1]["birth"])
    np.testing.assert_array_equal(a[1]["s"], b[1]["s"])
    np.testing.assert_allclose(b[2], a[2], rtol=1e-9, atol=1e-11 * np.abs(a[2]).max())
    diag, back = retouch_kinds(b[0], 256, 3)
    assert diag > 0 and back > 0


def test_mixed_lu_form_follows_the_oracle():
    ch = configs.cube8(K=64.0, k_max=32, capacity=256)
    cfg = configs.synthetic_configuration(ch, 200, seed=3)
    oc = oracle_for(ch, p_insert=0.4, p_flip=0.3)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    with pk.Context([ch], precision=pk.CTAUX_MIXED, trace_capacity=4 * 32, p_insert=0.4,
                    p_flip=0.3, refresh_every=8, gamma_form=pk.ctaux.CTAUX_GAMMA_LU) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.sweep(4)
        ctx.synchronize()
        tr = ctx.trace(0)
        recs = oc.run(len(tr))   # near ties end blocks early (decided in FP64)
        compare_traces(tr, recs, RTOL_MIXED)
        compare_config(ctx, 0, oc)


def test_gamma_form_is_validated():
    ch = configs.cube8(K=4.0, k_max=8, capacity=64)
    with pytest.raises(pk.CtauxError):
        pk.Context([ch], gamma_form=2)
