"""Failure reporting on the GPU without a GPU fault (needs a GB300).

  * Drift: a from-scratch recomputation whose relative drift
    max |N_run - N_fresh| / max |N_fresh| is above the context's drift_limit
    makes the next synchronous call return CTAUX_EDRIFT once; the chain goes on
    from the fresh N and still follows the oracle.
  * Bounded waits of the tensor-core flush: with the test setting of
    tc_wait_limit the MMA issuer waits on a barrier that nothing completes; the
    wait runs out, the kernel drains its copies, frees its tensor memory and
    returns, and the host reads CTAUX_ETIMEOUT.  The device stays usable.
"""
import pytest

from parity import compare_config, compare_traces, oracle_for
from workloads import configs

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1010_3690_gb300")


def test_drift_limit_reports_edrift_once_and_chain_continues():
    ch = configs.cube8(K=256.0, k_max=64, capacity=1024)
    cfg = configs.synthetic_configuration(ch, 430, seed=3)
    with pk.Context([ch], precision=pk.CTAUX_MIXED, refresh_every=0, drift_limit=1e-9,
                    trace_capacity=4096) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])  # no report
        ctx.sweep(24)
        with pytest.raises(pk.CtauxError) as ei:
            ctx.recompute()
        assert ei.value.code == 6                      # CTAUX_EDRIFT
        st = ctx.stats(0)
        assert st["last_drift_rel"] > 1e-9 and st["refreshes"] >= 1
        ctx.sweep(2)
        ctx.synchronize()                              # reported once
        tr = ctx.trace(0)
        oc = oracle_for(ch)
        oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        # 24 blocks without a refresh: float32 ratio errors grow to ~1e-5 (the
        # decisions are protected by the near-tie guard)
        compare_traces(tr, oc.run(len(tr)), 1e-4)
        compare_config(ctx, 0, oc)


def test_fp64_refresh_drift_below_1e8_relative():
    """The FP64 form's running N stays within 1e-8 (relative) of the from-scratch
    N over 48 blocks without a refresh: no CTAUX_EDRIFT at that limit."""
    ch = configs.cube8(K=256.0, k_max=64, capacity=1024)
    cfg = configs.synthetic_configuration(ch, 430, seed=3)
    with pk.Context([ch], refresh_every=0, drift_limit=1e-8) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.sweep(48)
        ctx.recompute()
        assert ctx.stats(0)["last_drift_rel"] < 1e-8


def test_flush_wait_that_runs_out_returns_etimeout():
    ch = configs.cube8(K=256.0, k_max=64, capacity=1024)
    cfg = configs.synthetic_configuration(ch, 430, seed=3)
    with pk.Context([ch], precision=pk.CTAUX_MIXED, refresh_every=0, tc_wait_limit=-2000) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.sweep(2)
        with pytest.raises(pk.CtauxError) as ei:
            ctx.synchronize()
        assert ei.value.code == 7                      # CTAUX_ETIMEOUT
        assert ctx.stats(0)["status"] & 8              # DS_TIMEOUT, read back from the device
    # the device is healthy: a normal context runs and follows the oracle
    with pk.Context([ch], precision=pk.CTAUX_MIXED, refresh_every=0, trace_capacity=256) as ctx:
        ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        ctx.sweep(2)
        ctx.synchronize()
        tr = ctx.trace(0)
        oc = oracle_for(ch)
        oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        compare_traces(tr, oc.run(len(tr)), 1e-5)
