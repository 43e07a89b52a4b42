"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test checks the oracle against a value the paper or the mathematics fixes:
published Philox vectors, operator-algebra traces (exact diagonalisation),
closed forms (first insertion, U -> 0), detailed balance of insertion/removal
and of spin-flip pairs driven through OracleChain.step with planted uniforms,
the determinant identities of Secs. III-IV, and the interacting impurity
solved by exact diagonalisation.  Planted mistakes in the oracle (move factors,
the equal-time convention) fail their pins.
"""
import math

import numpy as np
import pytest
from scipy import integrate, linalg, stats

from conftest import load_kat
from oracle import philox
from oracle.ctaux import FLIP, INSERT, REMOVE, OracleChain, cluster_momenta, matsubara
from oracle.ed import AndersonED, SingleSpinFreeED
from workloads import configs, g0tables


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    for rounds, ctr, key, want in load_kat():
        assert rounds == 10
        got = philox.philox4x32_10(ctr, key)[:, 0]
        assert [int(v) for v in got] == want


def test_uniform_mapping_range_and_resolution():
    u, v = philox.uniforms(0, 0, np.arange(100000), 0)
    assert u.min() >= 0.0 and u.max() < 1.0 and v.min() >= 0.0 and v.max() < 1.0
    # 53-bit mantissa: u * 2^53 is an integer
    assert np.all(np.floor(u * 2.0 ** 53) == u * 2.0 ** 53)
    # uniformity (KS) and independence of the two halves
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.02


# ---------------------------------------------------------------- tables
def test_semicircle_table_against_adaptive_quadrature():
    beta = 10.0
    tab = g0tables.semicircle_g0(beta, 1001)
    assert tab[0] == pytest.approx(-0.5, abs=1e-12)      # G0(0+) = -(1 - n0), n0 = 1/2
    assert tab[-1] == pytest.approx(-0.5, abs=1e-12)     # G0(beta-) = -n0
    for j in (10, 250, 500, 900):
        tau = j * beta / 1000

        def f(e):
            rho = 2.0 / (math.pi * 4.0) * math.sqrt(max(4.0 - e * e, 0.0))
            return rho * g0tables.fermion_g(e, tau, beta)[()]
        ref, _ = integrate.quad(f, -2.0, 2.0, limit=400, epsabs=1e-13)
        assert tab[j] == pytest.approx(ref, abs=1e-10)


def test_aim_table_against_matrix_exponential():
    beta = 5.0
    h = g0tables.aim_single_particle_h((-1.0, 0.0, 1.0), (0.5, 0.5, 0.5))
    tab = g0tables.aim_g0(beta, 101)
    for j in (1, 37, 99):
        tau = j * beta / 100
        # G0(tau) = -[e^{-tau h} (1 + e^{-beta h})^{-1}]_{00}
        ref = -(linalg.expm(-tau * h) @ np.linalg.inv(np.eye(4) + linalg.expm(-beta * h)))[0, 0]
        assert tab[j] == pytest.approx(ref, abs=1e-13)


def test_cluster_table_sum_rule_and_symmetry():
    ch = configs.cube8()
    g = ch.table[0]
    # local: G(0+) + G(beta-) = -1; half filling: G(0+) = -1/2
    assert g[0, 0] + g[0, -1] == pytest.approx(-1.0, abs=1e-12)
    assert g[0, 0] == pytest.approx(-0.5, abs=1e-12)
    # every displacement: G(0+) + G(beta-) = -delta_{dx,0} (anticommutator)
    assert np.allclose(g[1:, 0] + g[1:, -1], 0.0, atol=1e-12)


# ------------------------------------------- weight and estimator vs ED
def _aim_chain(beta=5.0, U=4.0, K=1.0, n_tau=20001, seed=0):
    ch = configs.aim_ed(beta=beta, U=U, K=K, n_tau=n_tau, seed=seed)
    return OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=seed)


def test_weight_equals_time_ordered_trace():
    """det N^{-1} = prod e^{V_i} <T prod e^{-V_i n(tau_i)}>_0 (Eq. Zn_div_Z0 with reading C4)."""
    oc = _aim_chain()
    ed = SingleSpinFreeED(oc.beta)
    rng = np.random.default_rng(3)
    for _ in range(12):
        n = int(rng.integers(1, 7))
        taus = rng.choice(oc.n_tau - 1, size=n, replace=False) * oc.dtau   # on the grid: exact
        s = rng.choice([-1, 1], size=n)
        site = np.zeros(n, np.int64)
        for spin in (0, 1):
            V = oc.gamma * (1.0 if spin == 0 else -1.0) * s
            det = np.linalg.det(oc.ninv(spin, taus, site, s))
            ref = np.prod(np.exp(V)) * ed.weight(taus, -V)
            assert det == pytest.approx(ref, rel=1e-11)


def test_green_estimator_equals_operator_trace():
    """G(a,b) = G0(a,b) + G0(a,l)[(e^V-1)N]_lm G0(m,b) equals the trace with the field (C9)."""
    oc = _aim_chain()
    ed = SingleSpinFreeED(oc.beta)
    rng = np.random.default_rng(4)
    for _ in range(4):
        n = int(rng.integers(1, 6))
        js = rng.choice(oc.n_tau - 1, size=n + 2, replace=False)
        taus = js[:n] * oc.dtau
        ta, tb = js[n] * oc.dtau, js[n + 1] * oc.dtau
        s = rng.choice([-1, 1], size=n)
        oc.set_config(taus, np.zeros(n, np.int64), s, np.arange(n), 0)
        for spin in (0, 1):
            N = oc.N(spin)
            M = (oc.exp_v(spin, s) - 1.0)[:, None] * N
            est = (oc.g0(spin, ta, 0, tb, 0) + oc.g0(spin, ta, 0, taus, 0) @ M
                   @ oc.g0(spin, taus, 0, tb, 0))
            V = oc.gamma * (1.0 if spin == 0 else -1.0) * s
            assert est == pytest.approx(ed.green(ta, tb, taus, -V), rel=1e-10, abs=1e-12)


def test_measure_G_matches_pointwise_estimator_and_sum_rule():
    ch = configs.cube8(K=4.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=1)
    oc.run(400)
    assert oc.order > 3
    G = oc.measure_G(n_bins=6, n_anchors=3)
    # recompute one class/bin by hand
    spin, x_a, c = 1, 3, 2
    tau_c = (c + 0.5) * oc.beta / 6
    N = oc.N(spin)
    M = (oc.exp_v(spin, oc.s) - 1.0)[:, None] * N
    acc = 0.0
    for j in range(3):
        tb = j * oc.beta / 3
        ta = tb + tau_c
        sg = 1.0
        if ta >= oc.beta:
            ta, sg = ta - oc.beta, -1.0
        est = (oc.g0(spin, ta, x_a, tb, 0) + oc.g0(spin, ta, x_a, oc.tau, oc.site) @ M
               @ oc.g0(spin, oc.tau, oc.site, tb, 0))
        acc += sg * est / 3
    assert G[spin, ch.dx_class[x_a, 0], c] == pytest.approx(acc, rel=1e-12)
    # per configuration, local G(0+) + G(beta-) = -1 (antiperiodicity of G0)
    for spin in (0, 1):
        tb = 0.7
        eps = 1e-9
        vals = []
        for ta in (tb + eps, tb + oc.beta - eps):
            sg = 1.0
            if ta >= oc.beta:
                ta, sg = ta - oc.beta, -1.0
            M = (oc.exp_v(spin, oc.s) - 1.0)[:, None] * oc.N(spin)
            vals.append(sg * (oc.g0(spin, ta, 0, tb, 0) + oc.g0(spin, ta, 0, oc.tau, oc.site)
                              @ M @ oc.g0(spin, oc.tau, oc.site, tb, 0)))
        assert vals[0] + vals[1] == pytest.approx(-1.0, abs=1e-6)


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("maker", ["aim1", "cube8"])
def test_first_insertion_closed_form(maker):
    """Half filling, particle-hole symmetric G0: R(0 -> 1) = K + beta U N_c / 4 for either s."""
    ch = configs.aim1(K=1.0) if maker == "aim1" else configs.cube8(K=3.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=0)
    want = ch.K + ch.beta * ch.U * ch.n_c / 4.0
    seen = 0
    while seen < 4:
        oc2 = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=oc.seed)
        oc2.t = oc.t
        rec = oc2.step()
        if rec["move"] == INSERT:
            assert rec["R"] == pytest.approx(want, rel=1e-12)
            seen += 1
        oc.t += 1


def _plant(oc, script):
    """Replace the Philox draws of proposals t in `script` by the given uniforms
    (u_move, u_acc, u_tau, u_site, u_spin, u_idx); other proposals keep theirs."""
    drawn = oc.draws
    oc.draws = lambda t: script[t] if t in script else drawn(t)


def _u_insert(oc):
    return 0.5 * oc.p_insert


def _u_remove(oc):
    return oc.p_insert + 0.5 * oc.p_remove


def _u_flip(oc):
    return oc.p_insert + oc.p_remove + 0.5 * oc.p_flip


def _u_pick(i, n):
    """u with floor(u n) = i: the i-th interacting vertex in birth order."""
    return (i + 0.5) / n


def _insert_then_remove(oc, u_tau, u_site, u_spin):
    """Drive OracleChain.step through an accepted insertion and the removal of the
    same vertex (u_acc = 0 accepts any |R| > 0).  Returns both trace records."""
    n, t = oc.order, oc.t
    _plant(oc, {t: (_u_insert(oc), 0.0, u_tau, u_site, u_spin, 0.5),
                t + 1: (_u_remove(oc), 0.0, 0.5, 0.5, 0.5, _u_pick(n, n + 1))})
    return oc.step(), oc.step()


def _flip_twice(oc, i):
    n, t = oc.order, oc.t
    u = (_u_flip(oc), 0.0, 0.5, 0.5, 0.5, _u_pick(i, n))
    _plant(oc, {t: u, t + 1: u})
    return oc.step(), oc.step()


def test_insert_remove_detailed_balance():
    """An accepted insertion c -> c' and the removal of the same vertex c' -> c,
    both through OracleChain.step: R_ins(c -> c') R_rem(c' -> c) = 1 (Eq. insprob
    and its inverse move), and the chain returns to c with its determinants."""
    ch = configs.cube8(K=2.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=5)
    oc.run(300)
    assert oc.order > 2
    rng = np.random.default_rng(0)
    for _ in range(5):
        before = (oc.tau.copy(), oc.s.copy(), list(oc._logdet))
        n = oc.order
        r_ins, r_rem = _insert_then_remove(oc, *rng.uniform(0.0, 1.0, 3))
        assert r_ins["move"] == INSERT and r_rem["move"] == REMOVE
        assert r_ins["accept"] and r_rem["accept"] and r_rem["birth"] == r_ins["birth"]
        assert r_ins["n"] == n and r_rem["n"] == n + 1
        assert r_ins["R"] * r_rem["R"] == pytest.approx(1.0, rel=1e-10)
        np.testing.assert_array_equal(oc.tau, before[0])
        np.testing.assert_array_equal(oc.s, before[1])
        assert oc._logdet == pytest.approx(before[2], rel=1e-12, abs=1e-10)


def test_flip_pair_detailed_balance():
    """A spin flip and the flip back, through OracleChain.step with p_flip > 0:
    R_flip(c -> c') R_flip(c' -> c) = 1, and each flip ratio is the ratio of the
    two configurations' dense determinants."""
    ch = configs.cube8(K=2.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=6, p_insert=0.4,
                     p_flip=0.3)
    oc.run(300)
    n = oc.order
    assert n > 4
    for i in (0, n // 2, n - 1):
        s_before = oc.s.copy()
        r1, r2 = _flip_twice(oc, i)
        assert r1["move"] == FLIP and r2["move"] == FLIP
        assert r1["accept"] and r2["accept"] and r1["birth"] == r2["birth"] == oc.birth[i]
        assert r1["s_new"] == -s_before[i] and r2["s_new"] == s_before[i]
        assert r1["R"] * r2["R"] == pytest.approx(1.0, rel=1e-10)
        np.testing.assert_array_equal(oc.s, s_before)
        s2 = s_before.copy()
        s2[i] = -s2[i]
        want = 1.0
        for spin in (0, 1):
            A0 = oc.ninv(spin, oc.tau, oc.site, s_before)
            A1 = oc.ninv(spin, oc.tau, oc.site, s2)
            want *= np.linalg.det(A1) / np.linalg.det(A0)
        assert r1["R"] == pytest.approx(want, rel=1e-9)


def test_flip_ratio_equals_ratio_of_operator_traces():
    """The flip branch's R against exact diagonalisation: det N^{-1} =
    prod e^{V_i} <T prod e^{-V_i n(tau_i)}>_0 per spin (Eq. Zn_div_Z0), so a flip of
    vertex i changes the weight by the ratio of two operator traces."""
    ch = configs.aim_ed(beta=5.0, U=4.0, K=1.0, n_tau=20001)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, p_insert=0.3, p_flip=0.4)
    ed = SingleSpinFreeED(oc.beta)
    rng = np.random.default_rng(8)
    for _ in range(4):
        n = int(rng.integers(2, 6))
        taus = rng.choice(oc.n_tau - 1, size=n, replace=False) * oc.dtau   # on the grid: exact
        s = rng.choice([-1, 1], size=n)
        oc.set_config(taus, np.zeros(n, np.int64), s, np.arange(n), 100)
        i = int(rng.integers(n))
        _plant(oc, {100: (_u_flip(oc), 0.0, 0.5, 0.5, 0.5, _u_pick(i, n))})
        rec = oc.step()
        s2 = s.copy()
        s2[i] = -s2[i]
        want = 1.0
        for spin in (0, 1):
            sig = 1.0 if spin == 0 else -1.0
            V0, V1 = oc.gamma * sig * s, oc.gamma * sig * s2
            w0 = np.prod(np.exp(V0)) * ed.weight(taus, -V0)
            w1 = np.prod(np.exp(V1)) * ed.weight(taus, -V1)
            want *= w1 / w0
        assert rec["move"] == FLIP and rec["birth"] == i
        assert rec["R"] == pytest.approx(want, rel=1e-10)


def test_removal_from_empty_configuration_rejects():
    """n = 0: a removal (or flip) is rejected without a ratio, the counter advances
    and the configuration stays empty (reading C7)."""
    ch = configs.cube8(K=2.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, p_insert=0.4, p_flip=0.3)
    for u_move in (_u_remove(oc), _u_flip(oc)):
        t = oc.t
        _plant(oc, {t: (u_move, 0.0, 0.5, 0.5, 0.5, 0.5)})
        rec = oc.step()
        assert not rec["accept"] and rec["birth"] == -1 and rec["R"] == 0.0
        assert oc.t == t + 1 and oc.order == 0


@pytest.mark.parametrize("p_flip", [0.0, 0.3])
def test_U_to_zero_limit(p_flip):
    """U -> 0: gamma -> 0, every determinant ratio (insertion, removal and spin
    flip) is 1, G = G0, and n ~ Poisson(K) whatever share of the moves are flips."""
    ch = configs.cube8(K=3.0)
    p_ins = 0.5 * (1.0 - p_flip)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, 0.0, ch.K, seed=2, p_insert=p_ins,
                     p_flip=p_flip)
    assert oc.gamma == 0.0
    orders = []
    n_flips = 0
    for _ in range(600 if p_flip == 0.0 else 900):
        for rec in oc.run(8):
            if rec["n"] > 0 or rec["move"] == INSERT:
                assert rec["ratio"][0] == pytest.approx(1.0, abs=1e-12)
                assert rec["ratio"][1] == pytest.approx(1.0, abs=1e-12)
                n_flips += rec["move"] == FLIP and rec["accept"]
        orders.append(oc.order)
    assert (n_flips > 500) == (p_flip > 0.0)
    G = oc.measure_G(n_bins=5, n_anchors=2)
    tau_c = (np.arange(5) + 0.5) * oc.beta / 5
    for cls in range(ch.n_c):
        x_a = int(np.where(ch.dx_class[:, 0] == cls)[0][0])
        ref = oc.g0(0, tau_c, x_a, 0.0, 0)
        assert np.allclose(G[0, cls], ref, atol=1e-8)
    orders = np.array(orders[100:])
    assert abs(orders.mean() - oc.K) < 0.5
    assert abs(orders.var() - oc.K) < 1.0


# ------------------------------------------ determinant identities (Sec. III)
def _config_with_preinserted(seed=9):
    ch = configs.cube8(K=2.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=seed)
    oc.run(300)
    return ch, oc


def test_single_change_ratio_identity():
    """LU ratio of a single spin change = 1 + lambda (1 - G_pp), G = N G0 (Eq. Akp1Ak, reading C2)."""
    ch, oc = _config_with_preinserted()
    n = oc.order
    for p in (0, n // 2, n - 1):
        s2 = oc.s.copy()
        s2[p] = -s2[p]
        for spin in (0, 1):
            N = oc.N(spin)
            G0 = oc.g0(spin, oc.tau[:, None], oc.site[:, None], oc.tau[None, :], oc.site[None, :])
            G = N @ G0
            sig = 1.0 if spin == 0 else -1.0
            lam = math.exp(oc.gamma * sig * (s2[p] - oc.s[p])) - 1.0
            s1, l1 = oc.slogdet(spin, oc.tau, oc.site, oc.s)
            s_2, l2 = oc.slogdet(spin, oc.tau, oc.site, s2)
            assert s1 * s_2 * math.exp(l2 - l1) == pytest.approx(1.0 + lam * (1.0 - G[p, p]),
                                                                 rel=1e-9)


def test_multi_change_ratio_equals_prod_lambda_det_gamma():
    """det A'/det A = prod_j (-lambda_j) det Gamma, Gamma = G0_PP - diag((1+lambda)/lambda) (Sec. III C)."""
    ch, oc = _config_with_preinserted()
    n = oc.order
    rng = np.random.default_rng(1)
    # append three s=0 vertices (pre-insertion) and change a mix of old and new spins
    tau = np.append(oc.tau, rng.uniform(0, oc.beta, 3))
    site = np.append(oc.site, rng.integers(0, ch.n_c, 3))
    s0 = np.append(oc.s, [0, 0, 0])
    P = [n, 1, n + 2, n // 2]
    s1 = s0.copy()
    s1[n], s1[1], s1[n + 2], s1[n // 2] = 1, 0, -1, -s0[n // 2]
    for spin in (0, 1):
        sig = 1.0 if spin == 0 else -1.0
        A0 = oc.ninv(spin, tau, site, s0)
        N = np.linalg.inv(A0)
        G0 = oc.g0(spin, tau[:, None], site[:, None], tau[None, :], site[None, :])
        G = N @ G0
        lam = np.array([math.exp(oc.gamma * sig * (s1[p] - s0[p])) - 1.0 for p in P])
        Gam = G[np.ix_(P, P)] - np.diag((1.0 + lam) / lam)
        direct = np.linalg.det(oc.ninv(spin, tau, site, s1)) / np.linalg.det(A0)
        assert direct == pytest.approx(np.prod(-lam) * np.linalg.det(Gam), rel=1e-9)
        # Woodbury flush (Eq. Nshermanmorrison): N' = D^{-1}(N - G_{:,P} Gamma^{-1} N_{P,:})
        D = np.ones(len(tau))
        D[P] = 1.0 + lam
        Nw = (N - G[:, P] @ np.linalg.inv(Gam) @ N[P, :]) / D[:, None]
        assert np.allclose(Nw, np.linalg.inv(oc.ninv(spin, tau, site, s1)), rtol=1e-8,
                           atol=1e-9 * np.abs(Nw).max())
        # deleting the s=0 rows and columns of N' gives N of the reduced configuration (Sec. IV C)
        keep = s1 != 0
        Nred = np.linalg.inv(oc.ninv(spin, tau[keep], site[keep], s1[keep]))
        assert np.allclose(Nw[np.ix_(keep, keep)], Nred, rtol=1e-8, atol=1e-9 * np.abs(Nred).max())


# ------------------------------------------ Matsubara / momentum estimator
def _simpson(f, x):
    """Composite Simpson along the last axis (odd number of equally spaced points)."""
    h = x[1] - x[0]
    return (h / 3.0) * (f[..., 0] + f[..., -1] + 4.0 * f[..., 1:-1:2].sum(-1) + 2.0 * f[..., 2:-1:2].sum(-1))


def test_g0_matsubara_against_quadrature_and_lehmann():
    """The tabulated G0's transform: Simpson per table interval against an independent
    fine quadrature of the interpolated G0 (C4, C20), and against the exact Lehmann
    sum of the impurity (table interpolation error only)."""
    oc = _aim_chain(n_tau=4001)
    F = 6
    w = matsubara(oc.beta, F)
    g = oc.g0_matsubara(F)[0, 0]
    tq = np.linspace(0.0, oc.beta, 300001)[1:-1]
    vals = oc.g0(0, tq, np.zeros_like(tq, dtype=np.int64), 0.0, 0)
    ref = np.trapezoid(np.exp(1j * w[:, None] * tq[None, :]) * vals[None, :], tq, axis=1)
    assert np.allclose(g, ref, rtol=1e-6, atol=1e-7), (g, ref)
    ed = SingleSpinFreeED(oc.beta)
    assert np.allclose(g, ed.g0_matsubara(w), rtol=1e-5, atol=1e-6)


def test_matsubara_estimator_is_fourier_transform_of_tau_estimator():
    """C20 against the C9 estimator: the Fourier integrals of G0(tau - tau_l) and
    G0(tau_m - tau') are done by quadrature of the tau-space G0 (split at the
    jump), then assembled as (1/beta) sum_lm u_xl M_lm v_my; the estimator's closed
    form (phases e^{+-iw tau} times G0(iw)) must agree.  A conjugated phase fails."""
    ch = configs.cube8(K=4.0, k_max=16, capacity=128)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=3)
    cfg = configs.synthetic_configuration(ch, 10, seed=5)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    F, n, n_c, beta = 3, oc.order, oc.n_c, oc.beta
    w = matsubara(beta, F)
    got = oc.measure_G_matsubara(F)
    g0_iw = oc.g0_matsubara(F)
    xs = np.arange(n_c)
    for spin in (0, 1):
        u = np.zeros((n_c, n, F), complex)     # int e^{iw tau} G0(x - x_l, tau - tau_l) dtau
        v = np.zeros((n, n_c, F), complex)     # int e^{-iw t} G0(x_m - y, tau_m - t) dt
        for l in range(n):
            for lo, hi in ((0.0, oc.tau[l]), (oc.tau[l], beta)):
                t = np.linspace(lo, hi, 20001)[None, :]
                inner = t[:, 1:-1]
                gu = oc.g0(spin, inner, xs[:, None], oc.tau[l], oc.site[l])      # [n_c, pts]
                gv = oc.g0(spin, oc.tau[l], oc.site[l], inner, xs[:, None])      # [n_c, pts]
                # endpoints: the one-sided limits of the piece
                eps = 1e-12 * beta
                e_lo = np.full((n_c, 1), lo + eps)
                e_hi = np.full((n_c, 1), hi - eps)
                gu = np.concatenate([oc.g0(spin, e_lo, xs[:, None], oc.tau[l], oc.site[l]), gu,
                                     oc.g0(spin, e_hi, xs[:, None], oc.tau[l], oc.site[l])], axis=1)
                gv = np.concatenate([oc.g0(spin, oc.tau[l], oc.site[l], e_lo, xs[:, None]), gv,
                                     oc.g0(spin, oc.tau[l], oc.site[l], e_hi, xs[:, None])], axis=1)
                tt = t[0]
                u[:, l, :] += _simpson(np.exp(1j * w[None, :, None] * tt) * gu[:, None, :], tt)
                v[l, :, :] += _simpson(np.exp(-1j * w[None, :, None] * tt) * gv[:, None, :], tt)
        M = (oc.exp_v(spin, oc.s) - 1.0)[:, None] * oc.N(spin)
        ref = g0_iw[spin][oc.dx_class] + np.einsum("xlf,lm,myf->xyf", u, M, v) / beta
        assert np.allclose(got[spin], ref, rtol=1e-6, atol=1e-8), np.abs(got[spin] - ref).max()
        # the closed form of one factor, and a planted conjugated phase
        G0xy = g0_iw[spin][oc.dx_class]
        u_closed = G0xy[:, oc.site, :] * np.exp(1j * w[None, None, :] * oc.tau[None, :, None])
        assert np.allclose(u, u_closed, rtol=1e-6, atol=1e-9)
        u_bad = G0xy[:, oc.site, :] * np.exp(-1j * w[None, None, :] * oc.tau[None, :, None])
        bad = G0xy + np.einsum("xlf,lm,myf->xyf", u_bad, M, v) / beta
        assert np.abs(bad - ref).max() > 1e3 * np.abs(got[spin] - ref).max() + 1e-6


def test_cluster_momenta_of_the_free_cluster():
    """With no vertices the estimator is G0; its cluster-momentum transform equals the
    coarse-grained lattice sum (1/N_p) sum_k~ 1/(iw - eps(K + k~)) that generated the
    table (cube8, half filling), up to the table's interpolation error."""
    ch = configs.cube8(K=4.0, k_max=16, capacity=128)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=0)
    F = 5
    w = matsubara(oc.beta, F)
    G = oc.measure_G_matsubara(F)                      # n = 0: G = G0
    cl = configs.cluster(8)
    GK = cluster_momenta(G, cl.sites, cl.K)            # [2, n_K, F]
    kt = g0tables._patch_offsets(cl, 12)
    for iK, K in enumerate(cl.K):
        xi = g0tables.dispersion(K[None, :] + kt)      # mu = 0 at half filling
        ref = (1.0 / (1j * w[None, :] - xi[:, None])).mean(axis=0)
        for spin in (0, 1):
            assert np.allclose(GK[spin, iK], ref, rtol=2e-5, atol=1e-6), (iK, GK[spin, iK], ref)
    # and back: sum_K e^{iK.(r_x - r_y)} G(K) / N_c returns G_xy
    ph = np.exp(1j * (cl.sites.astype(float) @ cl.K.T))
    back = np.einsum("xk,skf,yk->sxyf", ph, GK, ph.conj()) / 8
    assert np.allclose(back, G, atol=1e-12)


# ------------------------------------------------------- interacting ED
@pytest.mark.slow
def test_oracle_montecarlo_matches_exact_diagonalisation():
    """Anderson impurity + 3 bath levels: <order> = K + beta U (1/2 - d), and G(tau) and
    G(iw_n) vs ED."""
    beta, U, K = 5.0, 4.0, 1.0
    ch = configs.aim_ed(beta=beta, U=U, K=K, n_tau=4001)
    oc = OracleChain(ch.table, ch.dx_class, beta, U, K, seed=11)
    ed = AndersonED(beta, U)
    d = ed.double_occupancy()
    nb, n_batch, per_batch, k = 10, 12, 160, 8
    F = 4
    g0_iw = oc.g0_matsubara(F)
    oc.run(1500)
    Gs, orders, Gw = [], [], []
    for _ in range(n_batch):
        acc = np.zeros((2, 1, nb))
        accw = np.zeros((2, F), complex)
        o = 0.0
        for _ in range(per_batch):
            oc.run(k)
            acc += oc.measure_G(nb, 16)
            accw += oc.measure_G_matsubara(F, g0_iw)[:, 0, 0, :]
            o += oc.order
        Gs.append(acc / per_batch)
        Gw.append(accw / per_batch)
        orders.append(o / per_batch)
    Gs = np.array(Gs)
    mean = Gs.mean(axis=0)
    err = Gs.std(axis=0, ddof=1) / math.sqrt(n_batch)
    tc = (np.arange(nb) + 0.5) * beta / nb
    ref = ed.G(tc)
    z = (mean[:, 0, :] - ref[None, :]) / err[:, 0, :]
    assert np.all(np.abs(z) < 4.0), z
    chi2 = float(np.sum(z ** 2))
    assert chi2 < stats.chi2.ppf(0.999, z.size), chi2
    o_mean = np.mean(orders)
    o_err = np.std(orders, ddof=1) / math.sqrt(n_batch)
    assert abs(o_mean - (K + beta * U * (0.5 - d))) < 4.0 * o_err + 0.05
    # Matsubara estimator (C20) against the Lehmann sum, real and imaginary parts
    Gw = np.array(Gw)
    ref_w = ed.G_matsubara(matsubara(beta, F))
    for part in (np.real, np.imag):
        m_w = part(Gw).mean(axis=0)
        e_w = part(Gw).std(axis=0, ddof=1) / math.sqrt(n_batch)
        zw = (m_w - part(ref_w)[None, :]) / np.maximum(e_w, 1e-12)
        assert np.all(np.abs(zw) < 4.0), zw


# -------------------------------------------- planted mistakes are caught
def test_planted_equal_time_mistake_fails_weight_pin():
    """Using G0(0+) on the diagonal instead of G0(0-) must break the ED weight pin."""
    oc = _aim_chain()
    ed = SingleSpinFreeED(oc.beta)
    taus = np.array([40, 4000, 12000]) * oc.dtau
    s = np.array([1, -1, 1])
    site = np.zeros(3, np.int64)
    V = oc.gamma * s
    good = np.linalg.det(oc.ninv(0, taus, site, s))
    ref = np.prod(np.exp(V)) * ed.weight(taus, -V)
    assert good == pytest.approx(ref, rel=1e-11)
    A = oc.ninv(0, taus, site, s)
    ev = oc.exp_v(0, s)
    wrong_diag = oc.table[0, 0, 0]          # G0(0+) instead of G0(0-)
    A_bad = A.copy()
    for i in range(3):
        A_bad[i, i] = ev[i] - wrong_diag * (ev[i] - 1.0)
    assert abs(np.linalg.det(A_bad) / ref - 1.0) > 1e-3


@pytest.mark.parametrize("wrong", ["removal_post_move_order", "insertion_pre_move_order"])
def test_planted_move_factor_mistake_fails_detailed_balance(wrong):
    """A move factor taken at the wrong order (n - 1 after a removal, or n before
    an insertion), planted in the oracle, breaks R_ins R_rem = 1 through step()."""
    ch = configs.cube8(K=2.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=5)
    oc.run(300)
    right = oc.move_factor

    def planted(move, n):
        if wrong == "removal_post_move_order" and move == REMOVE:
            return (n - 1) / oc.K
        if wrong == "insertion_pre_move_order" and move == INSERT:
            return oc.K / n
        return right(move, n)
    oc.move_factor = planted
    r_ins, r_rem = _insert_then_remove(oc, 0.3, 0.6, 0.2)
    assert r_ins["accept"] and r_rem["accept"]
    assert abs(r_ins["R"] * r_rem["R"] - 1.0) > 1e-3


def test_planted_flip_factor_mistake_fails_flip_balance():
    """A flip that reuses the removal factor n/K, planted in the oracle, breaks
    R_flip R_flip' = 1."""
    ch = configs.cube8(K=2.0)
    oc = OracleChain(ch.table, ch.dx_class, ch.beta, ch.U, ch.K, seed=6, p_insert=0.4,
                     p_flip=0.3)
    oc.run(300)
    right = oc.move_factor
    oc.move_factor = lambda move, n: n / oc.K if move == FLIP else right(move, n)
    r1, r2 = _flip_twice(oc, oc.order // 2)
    assert abs(r1["R"] * r2["R"] - 1.0) > 1e-3
