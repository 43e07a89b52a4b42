"""Helpers shared by the GPU parity tests: run the oracle on the same proposals."""
import numpy as np

from oracle.ctaux import OracleChain


def oracle_for(ch, p_insert=0.5, p_flip=0.0):
    return OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=ch.seed,
                       chain_id=ch.chain_id, p_insert=p_insert, p_flip=p_flip)


def compare_traces(gpu, recs, rtol):
    """Per proposal: same counter, move, vertex, proposed spin and accept decision;
    determinant ratios within rtol (relative, absolute below 1).  Returns the largest
    relative ratio error seen."""
    assert len(gpu) == len(recs), (len(gpu), len(recs))
    worst = 0.0
    for g, o in zip(gpu, recs):
        assert int(g["t"]) == o["t"], (g, o)
        assert int(g["move"]) == o["move"], (g, o)
        assert int(g["n"]) == o["n"], (g, o)
        assert int(g["birth"]) == o["birth"], (g, o)
        assert int(g["s_new"]) == o["s_new"], (g, o)
        assert bool(int(g["accept"]) & 1) == o["accept"], (g, o)
        if o["birth"] < 0:
            continue
        for s in (0, 1):
            ref = o["ratio"][s]
            err = abs(g["ratio"][s] - ref) / max(1.0, abs(ref))
            worst = max(worst, err)
            assert err <= rtol, (s, g, o, err)
        err = abs(g["R"] - o["R"]) / max(1.0, abs(o["R"]))
        assert err <= rtol * 4, (g, o)
    return worst


def compare_config(ctx, chain, oc):
    cfg = ctx.get_config(chain)
    assert cfg["t"] == oc.t
    assert len(cfg["tau"]) == oc.order
    np.testing.assert_array_equal(cfg["birth"], oc.birth)
    np.testing.assert_array_equal(cfg["tau"], oc.tau)
    np.testing.assert_array_equal(cfg["site"], oc.site)
    np.testing.assert_array_equal(cfg["s"], oc.s)
    return cfg
