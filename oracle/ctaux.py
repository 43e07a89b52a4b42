"""Plain CT-AUX Markov chain: the oracle for the submatrix-update hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check of __graft_entry__ and
the CPU-baseline leg of bench.py may import this module.  The CUDA path never
calls it, and it shares no code with the CUDA path.

The submatrix update (paper Secs. III-IV) is an exact rearrangement of plain
CT-AUX ("mathematically equivalent", Sec. VI).  So this oracle is the plain
definition of the random walk of Sec. II B, with no Gamma matrix, no Woodbury
formula and no s=0 vertices:

  * weight of a configuration {(tau_i, x_i, s_i)} (Eq. Zn_div_Z0, Eq. Nmatrix):
        prod_sigma det N_sigma^{-1},
        N_sigma^{-1} = e^{V_sigma} - G0_sigma (e^{V_sigma} - 1),
        e^{V_sigma} = diag(exp(gamma * sigma * s_i)), sigma = +1 (up), -1 (down);
  * cosh(gamma) = 1 + beta U N_c / (2K) (Eq. gamma, with the site sum of a
    cluster folded into the expansion constant);
  * insertion R = K/(n+1) prod_sigma det-ratio (Eq. insprob); removal
    R = n/K prod_sigma det-ratio (the inverse move); spin flip R = prod det-ratio;
  * accept iff u < min(1, |R|); the sign of R multiplies the walker's sign;
  * every determinant ratio is taken from two dense LU factorisations
    (numpy slogdet) of the full N^{-1} matrices.

Readings of the paper used here (it is silent or ambiguous on these):
  C1  e^{V_up} = e^{+gamma s}, e^{V_down} = e^{-gamma s}.
  C4  G0(tau) = -<T d(tau) d^dagger>; for tau<0, G0(tau) = -G0(tau+beta); equal
      times (including the diagonal) take G0(0-) = -G0(beta-).  Linear
      interpolation in the table: idx = floor(tau/dtau) clamped to n_tau-2,
      value = (1-f) T[idx] + f T[idx+1].
  C7  proposal t draws move (insert with p_insert, remove with p_remove, else
      flip); an insertion takes tau = u*beta, site = floor(u*N_c), s = +1 if
      u < 1/2 else -1; a removal or flip picks floor(u*n) in the order of birth
      (birth = index t of the insertion proposal); n = 0 rejects.
  C8  uniforms from Philox-4x32-10 keyed by (seed) with counter
      (t, chain, purpose); see oracle.philox.
  C9  G(dx, tau) estimator: G(a,b) = G0(a,b) + sum_lm G0(a,l) [(e^V-1)N]_lm G0(m,b),
      a = (x_a, tau_b + tau) and anchors b = (site 0, j beta / n_anchors).
  C20 Matsubara and cluster-momentum estimator (Sec. IV D: measure directly in
      cluster momenta and Matsubara frequencies): the Fourier transform
      (1/beta) int int dtau dtau' e^{i w (tau - tau')} of the C9 estimator,
          G_xy(iw) = G0_xy(iw) + (1/beta) sum_lm G0_{x x_l}(iw) e^{i w tau_l} M_lm
                                                 e^{-i w tau_m} G0_{x_m y}(iw),
      M = (e^V - 1) N, w_n = (2n+1) pi / beta, G0(iw) = int_0^beta e^{iw tau} G0(tau)
      of the same (interpolated) G0 the weights use; cluster momenta by
      G(K) = (1/N_c) sum_xy e^{-iK.(r_x - r_y)} G_xy.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox

INSERT, REMOVE, FLIP = 0, 1, 2
SIGMAS = (1.0, -1.0)


def matsubara(beta, n_freq):
    """Fermionic Matsubara frequencies w_n = (2n+1) pi / beta, n = 0 .. n_freq-1."""
    return (2.0 * np.arange(n_freq) + 1.0) * math.pi / float(beta)


def cluster_momenta(G_xy, sites, kvecs):
    """G(K) = (1/N_c) sum_xy e^{-i K.(r_x - r_y)} G_xy (C20).

    G_xy: [..., n_c, n_c, F]; sites: [n_c, d] positions; kvecs: [n_K, d].
    Returns [..., n_K, F]."""
    ph = np.exp(-1j * (np.asarray(kvecs, dtype=np.float64) @ np.asarray(sites, dtype=np.float64).T))
    n_c = ph.shape[1]
    return np.einsum("kx,...xyf,ky->...kf", ph, G_xy, ph.conj()) / n_c


class OracleChain:
    def __init__(self, table, dx_class, beta, U, K, seed=0, chain_id=0, p_insert=0.5,
                 p_flip=0.0):
        self.table = np.ascontiguousarray(table, dtype=np.float64)  # [2, n_classes, n_tau]
        self.dx_class = np.ascontiguousarray(dx_class, dtype=np.int64)
        self.n_c = self.dx_class.shape[0]
        self.n_tau = self.table.shape[2]
        self.beta = float(beta)
        self.U = float(U)
        self.K = float(K)
        self.dtau = self.beta / (self.n_tau - 1)
        self.gamma = math.acosh(1.0 + self.beta * self.U * self.n_c / (2.0 * self.K))
        self.seed = int(seed)
        self.chain_id = int(chain_id)
        self.p_insert = float(p_insert)
        self.p_flip = float(p_flip)
        self.p_remove = 1.0 - self.p_insert - self.p_flip
        self.tau = np.zeros(0)
        self.site = np.zeros(0, dtype=np.int64)
        self.s = np.zeros(0, dtype=np.int64)
        self.birth = np.zeros(0, dtype=np.int64)
        self.t = 0
        self.sign = 1.0
        self._logdet = [0.0, 0.0]
        self._sgndet = [1.0, 1.0]

    # ------------------------------------------------------------------ G0
    def _interp(self, spin, cls, x):
        """Linear interpolation of the table row cls at 0 <= x <= beta (C4)."""
        pos = x / self.dtau
        idx = np.floor(pos).astype(np.int64)
        idx = np.clip(idx, 0, self.n_tau - 2)
        f = pos - idx
        row = self.table[spin]
        return (1.0 - f) * row[cls, idx] + f * row[cls, idx + 1]

    def g0(self, spin, tau_i, x_i, tau_j, x_j):
        """G0_sigma(x_i - x_j, tau_i - tau_j) for broadcastable arrays (C4)."""
        tau_i, x_i, tau_j, x_j = np.broadcast_arrays(
            np.asarray(tau_i, dtype=np.float64), np.asarray(x_i, dtype=np.int64),
            np.asarray(tau_j, dtype=np.float64), np.asarray(x_j, dtype=np.int64))
        dt = tau_i - tau_j
        cls = self.dx_class[x_i, x_j]
        out = np.empty(dt.shape)
        pos = dt > 0.0
        neg = dt < 0.0
        eq = ~(pos | neg)
        out[pos] = self._interp(spin, cls[pos], dt[pos])
        out[neg] = -self._interp(spin, cls[neg], dt[neg] + self.beta)
        out[eq] = -self.table[spin, cls[eq], self.n_tau - 1]
        return out

    # ------------------------------------------------------------- N^{-1}
    def exp_v(self, spin, s):
        return np.exp(self.gamma * SIGMAS[spin] * np.asarray(s, dtype=np.float64))

    def ninv(self, spin, tau=None, site=None, s=None):
        """N_sigma^{-1} = e^V - G0 (e^V - 1) for a configuration (Eq. Nmatrix)."""
        if tau is None:
            tau, site, s = self.tau, self.site, self.s
        n = len(tau)
        if n == 0:
            return np.zeros((0, 0))
        G0 = self.g0(spin, tau[:, None], site[:, None], tau[None, :], site[None, :])
        ev = self.exp_v(spin, s)
        return np.diag(ev) - G0 * (ev - 1.0)[None, :]

    def slogdet(self, spin, tau, site, s):
        if len(tau) == 0:
            return 1.0, 0.0
        sg, ld = np.linalg.slogdet(self.ninv(spin, tau, site, s))
        return float(sg), float(ld)

    def N(self, spin):
        """Explicit N_sigma = inverse(N_sigma^{-1}) of the current configuration."""
        if len(self.tau) == 0:
            return np.zeros((0, 0))
        return np.linalg.inv(self.ninv(spin))

    # -------------------------------------------------------------- moves
    _DRAW_BLOCK = 512

    def draws(self, t):
        """The six uniforms of proposal t (drawn for 512 consecutive t at a time)."""
        base = (t // self._DRAW_BLOCK) * self._DRAW_BLOCK
        if getattr(self, "_draw_base", None) != base:
            ts = np.arange(base, base + self._DRAW_BLOCK, dtype=np.uint64)
            cols = []
            for purpose in (philox.PURPOSE_MOVE_ACCEPT, philox.PURPOSE_TAU_SITE,
                            philox.PURPOSE_SPIN_INDEX):
                cols.extend(philox.uniforms(self.seed, self.chain_id, ts, purpose))
            # order: u_move, u_accept, u_tau, u_site, u_spin, u_index
            self._draw_tab = np.stack(cols, axis=1)
            self._draw_base = base
        return tuple(float(v) for v in self._draw_tab[t - base])

    def move_factor(self, move, n):
        """Proposal-probability factor of a move from order n (Eq. insprob): an
        insertion picks tau, site and s with density K-normalised over n+1
        vertices, K/(n+1); a removal, its inverse from order n, n/K; a spin flip
        keeps n, 1."""
        if move == INSERT:
            return self.K / (n + 1)
        if move == REMOVE:
            return n / self.K
        return 1.0

    def step(self):
        """One Metropolis proposal (index self.t).  Returns its trace record."""
        t = self.t
        u_move, u_acc, u_tau, u_site, u_spin, u_idx = self.draws(t)
        n = len(self.tau)
        if u_move < self.p_insert:
            move = INSERT
        elif u_move < self.p_insert + self.p_remove:
            move = REMOVE
        else:
            move = FLIP
        rec = dict(t=t, move=move, n=n, u=u_acc)
        if move == INSERT:
            tau_new = u_tau * self.beta
            site_new = min(int(math.floor(u_site * self.n_c)), self.n_c - 1)
            s_new = 1 if u_spin < 0.5 else -1
            new = (np.append(self.tau, tau_new), np.append(self.site, site_new),
                   np.append(self.s, s_new), np.append(self.birth, t))
            f = self.move_factor(INSERT, n)
            rec.update(birth=t, s_new=s_new)
        else:
            if n == 0:
                self.t += 1
                rec.update(birth=-1, s_new=0, ratio=(0.0, 0.0), R=0.0, accept=False)
                return rec
            idx = min(int(math.floor(u_idx * n)), n - 1)
            rec.update(birth=int(self.birth[idx]))
            if move == REMOVE:
                keep = np.arange(n) != idx
                new = (self.tau[keep], self.site[keep], self.s[keep], self.birth[keep])
                f = self.move_factor(REMOVE, n)
                rec.update(s_new=0)
            else:
                s2 = self.s.copy()
                s2[idx] = -s2[idx]
                new = (self.tau, self.site, s2, self.birth)
                f = self.move_factor(FLIP, n)
                rec.update(s_new=int(s2[idx]))
        ratios = []
        dets = []
        for spin in (0, 1):
            sg, ld = self.slogdet(spin, new[0], new[1], new[2])
            dets.append((sg, ld))
            ratios.append(sg * self._sgndet[spin] * math.exp(ld - self._logdet[spin]))
        R = f * ratios[0] * ratios[1]
        accept = bool(u_acc < min(1.0, abs(R)))
        rec.update(ratio=(ratios[0], ratios[1]), R=R, accept=accept)
        if accept:
            self.tau, self.site, self.s, self.birth = new
            for spin in (0, 1):
                self._sgndet[spin], self._logdet[spin] = dets[spin]
            if R < 0:
                self.sign = -self.sign
        self.t += 1
        return rec

    def run(self, n_proposals):
        return [self.step() for _ in range(n_proposals)]

    # ------------------------------------------------------- checkpoints
    def set_config(self, tau, site, s, birth, t):
        order = np.argsort(np.asarray(birth), kind="stable")
        self.tau = np.asarray(tau, dtype=np.float64)[order]
        self.site = np.asarray(site, dtype=np.int64)[order]
        self.s = np.asarray(s, dtype=np.int64)[order]
        self.birth = np.asarray(birth, dtype=np.int64)[order]
        self.t = int(t)
        for spin in (0, 1):
            self._sgndet[spin], self._logdet[spin] = self.slogdet(spin, self.tau, self.site,
                                                                  self.s)

    @property
    def order(self):
        return len(self.tau)

    # -------------------------------------------------------- measurement
    def measure_G(self, n_bins, n_anchors):
        """Per-configuration G_sigma(dx class, tau bin centre), shape [2, n_classes, n_bins] (C9)."""
        n_classes = self.table.shape[1]
        out = np.zeros((2, n_classes, n_bins))
        cls_a = self.dx_class[:, 0]                          # class of (x_a - 0) per site x_a
        count = np.bincount(cls_a, minlength=n_classes).astype(np.float64)
        tau_c = (np.arange(n_bins) + 0.5) * self.beta / n_bins
        tau_b = np.arange(n_anchors) * self.beta / n_anchors
        # evaluation points a: [anchor, site, bin]
        shape = (n_anchors, self.n_c, n_bins)
        ta = np.broadcast_to(tau_b[:, None, None] + tau_c[None, None, :], shape)
        sgn = np.where(ta >= self.beta, -1.0, 1.0)
        ta = np.where(ta >= self.beta, ta - self.beta, ta)
        xa = np.broadcast_to(np.arange(self.n_c)[None, :, None], shape)
        tb = np.broadcast_to(tau_b[:, None, None], ta.shape)
        xb = np.zeros_like(xa)
        n = self.order
        for spin in (0, 1):
            val = self.g0(spin, ta, xa, tb, xb)
            if n > 0:
                N = self.N(spin)
                M = (self.exp_v(spin, self.s) - 1.0)[:, None] * N
                gb = self.g0(spin, self.tau[None, :], self.site[None, :], tau_b[:, None],
                             np.zeros((n_anchors, 1), np.int64))       # [anchor, m]
                v = gb @ M.T                                           # v_b = M g_b, [anchor, l]
                gal = self.g0(spin, ta[..., None], xa[..., None], self.tau, self.site)  # [A,S,B,l]
                val = val + np.einsum("asbl,al->asb", gal, v)
            val = sgn * val
            per_site = val.sum(axis=0) / n_anchors                     # [site, bin]
            for x in range(self.n_c):
                out[spin, cls_a[x]] += per_site[x] / count[cls_a[x]]
        return out

    def g0_matsubara(self, n_freq):
        """G0_sigma,class(iw_n) = int_0^beta e^{iw tau} G0(tau) dtau of the interpolated
        table, [2, n_classes, n_freq] complex (C20).  G0 is linear on every table
        interval, so Simpson's rule on each interval (its midpoint added) leaves
        only the (w dtau)^4 error of the smooth phase factor."""
        w = matsubara(self.beta, n_freq)
        t0 = np.arange(self.n_tau - 1) * self.dtau
        tm = t0 + 0.5 * self.dtau
        t1 = t0 + self.dtau
        T = self.table
        mid = 0.5 * (T[..., :-1] + T[..., 1:])
        e0, em, e1 = (np.exp(1j * w[:, None] * t[None, :]) for t in (t0, tm, t1))  # [F, n_tau-1]
        acc = (np.einsum("scj,fj->scf", T[..., :-1], e0) + 4.0 * np.einsum("scj,fj->scf", mid, em)
               + np.einsum("scj,fj->scf", T[..., 1:], e1))
        return acc * (self.dtau / 6.0)

    def measure_G_matsubara(self, n_freq, g0_iw=None):
        """Per-configuration G_sigma,xy(iw_n), [2, n_c, n_c, n_freq] complex (C20)."""
        if g0_iw is None:
            g0_iw = self.g0_matsubara(n_freq)
        w = matsubara(self.beta, n_freq)
        G0xy = g0_iw[:, self.dx_class, :]                         # [2, n_c, n_c, F]
        out = np.array(G0xy, dtype=np.complex128)
        n = self.order
        if n == 0:
            return out
        sel = np.zeros((self.n_c, n))
        sel[self.site, np.arange(n)] = 1.0                        # vertex l sits on site x_l
        ph = np.exp(1j * w[:, None] * self.tau[None, :])          # [F, n]
        for spin in (0, 1):
            M = (self.exp_v(spin, self.s) - 1.0)[:, None] * self.N(spin)
            # S_zw(iw) = sum_{l on z, m on w} e^{iw tau_l} M_lm e^{-iw tau_m}
            S = np.einsum("zl,fl,lm,fm,wm->zwf", sel, ph, M, ph.conj(), sel)
            G0s = G0xy[spin]
            out[spin] += np.einsum("xzf,zwf,wyf->xyf", G0s, S, G0s) / self.beta
        return out
