"""Rank-one and submatrix updates of CT-AUX on the host CPU (the paper's
comparison of Sec. V A, Figs. 2-3: submatrix updates about 8x faster than
rank-one updates on CPUs at expansion orders 512-2048, with k_max ~ 64-128).

This is the CPU half of that comparison for `bench.py --cpu-k-sweep`: both
algorithms in float64 with numpy (BLAS products), one chain, one thread.  It is
not the product path (the CUDA library is) and not the oracle (which recomputes
every determinant from scratch); it shares no code with either.

Both run the same Markov chain from the same draws: insertions and removals
(Eq. insprob and its inverse: R = K/(n+1) prod det-ratio, n/K prod det-ratio),
accept iff u < min(1, |R|), removal index floor(u n) in birth order, n = 0
rejects; weights det N_sigma^{-1}, N^{-1} = e^V - G0 (e^V - 1) (Eq. Nmatrix),
e^{V_up} = e^{+gamma s}, e^{V_down} = e^{-gamma s}, G0 linearly interpolated,
antiperiodic, equal times G0(0-) = -G0(beta-).

  * Rank one: N is kept explicitly; an insertion's ratio is the Schur
    complement d - c N b of the bordered N^{-1} (a matrix-vector product), a
    removal's is N_pp; an accepted move updates N by a rank-one product.
  * Submatrix (Secs. III-IV): k_max s=0 vertices pre-inserted, the rows of the
    extended N and the G columns of the new vertices by two products, each
    proposal grows Gamma^{-1} by partitioning, and N is updated once per block
    by the Woodbury formula with the s=0 rows and columns removed.
"""
from __future__ import annotations

import math
import time

import numpy as np

INSERT, REMOVE = 0, 1
SIGMAS = (1.0, -1.0)


class Model:
    """Table interpolation and the vertex factors of one chain's model."""

    def __init__(self, table, dx_class, beta, U, K):
        self.table = np.ascontiguousarray(table, dtype=np.float64)
        self.dx_class = np.ascontiguousarray(dx_class, dtype=np.int64)
        self.n_c = self.dx_class.shape[0]
        self.n_tau = self.table.shape[2]
        self.beta, self.K = float(beta), float(K)
        self.inv_dtau = (self.n_tau - 1) / self.beta
        self.gamma = math.acosh(1.0 + self.beta * float(U) * self.n_c / (2.0 * self.K))

    def g0(self, spin, ti, xi, tj, xj):
        """G0_sigma(x_i - x_j, tau_i - tau_j), broadcasting."""
        ti, xi, tj, xj = np.broadcast_arrays(np.asarray(ti, float), np.asarray(xi, np.int64),
                                             np.asarray(tj, float), np.asarray(xj, np.int64))
        dt = ti - tj
        flat = self.table[spin].reshape(-1)
        base = self.dx_class[xi, xj] * self.n_tau
        neg = dt < 0.0
        x = np.where(neg, dt + self.beta, dt) * self.inv_dtau
        idx = np.clip(np.floor(x).astype(np.int64), 0, self.n_tau - 2)
        f = x - idx
        lo = flat[base + idx]
        hi = flat[base + idx + 1]
        v = lo + f * (hi - lo)
        v = np.where(neg, -v, v)
        return np.where(dt == 0.0, -flat[base + self.n_tau - 1], v)

    def ev(self, spin, s):
        return np.exp(self.gamma * SIGMAS[spin] * np.asarray(s, float))


def numpy_draws(seed):
    """Six uniforms per proposal t (u_move, u_acc, u_tau, u_site, u_spin, u_idx)."""
    rng = np.random.default_rng(seed)
    cache = {}

    def draws(t):
        while t not in cache:
            base = len(cache)
            block = rng.random((4096, 6))
            for i in range(4096):
                cache[base + i] = tuple(block[i])
        return cache[t]
    return draws


class _Chain:
    def __init__(self, model, draws, p_insert=0.5):
        self.m, self.draws, self.p_insert = model, draws, p_insert
        self.tau = np.zeros(0)
        self.site = np.zeros(0, np.int64)
        self.s = np.zeros(0, np.int64)
        self.t = 0
        self.N = [np.zeros((0, 0)), np.zeros((0, 0))]
        self.trace = []

    def set_config(self, tau, site, s, t):
        self.tau = np.asarray(tau, float).copy()
        self.site = np.asarray(site, np.int64).copy()
        self.s = np.asarray(s, np.int64).copy()
        self.t = int(t)
        for spin in (0, 1):
            n = len(self.tau)
            G0 = self.m.g0(spin, self.tau[:, None], self.site[:, None], self.tau[None, :],
                           self.site[None, :])
            e = self.m.ev(spin, self.s)
            self.N[spin] = np.linalg.inv(np.diag(e) - G0 * (e - 1.0)[None, :]) if n else np.zeros((0, 0))

    def proposal(self, t):
        u_move, u_acc, u_tau, u_site, u_spin, u_idx = self.draws(t)
        move = INSERT if u_move < self.p_insert else REMOVE
        return move, u_acc, u_tau * self.m.beta, min(int(u_site * self.m.n_c), self.m.n_c - 1), \
            (1 if u_spin < 0.5 else -1), u_idx


class RankOne(_Chain):
    """Rank-one (fast) updates: one O(n^2) update per accepted proposal, in place
    through BLAS (dgemv, dger) on a capacity-sized Fortran array; vertices live
    in slots [0, n), a removal moves the last slot into the freed one, and a list
    keeps the birth order the proposals index."""

    def set_config(self, tau, site, s, t):
        from scipy.linalg import blas
        self.blas = blas
        super().set_config(tau, site, s, t)
        n = len(self.tau)
        self.n = n
        self.order = list(range(n))     # slots in birth order
        self.N = [np.asfortranarray(self.N[spin]) for spin in (0, 1)]
        self.cap = n
        self._grow()

    def _grow(self):
        """Capacity of 64 more slots (the BLAS calls run over the whole array, so
        it stays a little above the order)."""
        n, cap = self.n, self.cap + 64
        pad = lambda a, dt: np.concatenate([a[:n], np.zeros(cap - n, dt)])
        self.tau, self.site, self.s = pad(self.tau, float), pad(self.site, np.int64), pad(self.s, np.int64)
        for spin in (0, 1):
            F = np.zeros((cap, cap), order="F")
            F[:n, :n] = self.N[spin][:n, :n]
            self.N[spin] = F
        self.cap = cap

    def matrices(self):
        """N in birth order (for checks)."""
        o = np.array(self.order, np.int64)
        return [F[np.ix_(o, o)] for F in self.N]

    def config(self):
        o = np.array(self.order, np.int64)
        return self.tau[o], self.site[o], self.s[o]

    def step(self):
        blas, cap = self.blas, self.cap
        move, u, tau, site, s_new, u_idx = self.proposal(self.t)
        n = self.n
        rec = {"t": self.t, "move": move, "n": n}
        self.t += 1
        if move == INSERT:
            if n + 1 >= cap:
                self._grow()
                cap = self.cap
            f = self.m.K / (n + 1)
            parts = []
            for spin in (0, 1):
                e_new = float(self.m.ev(spin, s_new))
                b = np.zeros(cap)
                c = np.zeros(cap)
                e_old = self.m.ev(spin, self.s[:n])
                b[:n] = -self.m.g0(spin, self.tau[:n], self.site[:n], tau, site) * (e_new - 1.0)
                c[:n] = -self.m.g0(spin, tau, site, self.tau[:n], self.site[:n]) * (e_old - 1.0)
                d = e_new - float(self.m.g0(spin, tau, site, tau, site)) * (e_new - 1.0)
                Nb = blas.dgemv(1.0, self.N[spin], b)
                parts.append((d - c @ Nb, Nb, c))
            R = f * parts[0][0] * parts[1][0]
            rec["ratio"] = (parts[0][0], parts[1][0])
            acc = u < min(1.0, abs(R))
            if acc:
                for spin in (0, 1):
                    S, Nb, c = parts[spin]
                    F = self.N[spin]
                    cN = blas.dgemv(1.0, F, c, trans=1)
                    blas.dger(1.0 / S, Nb, cN, a=F, overwrite_a=1)
                    F[:n, n] = -Nb[:n] / S
                    F[n, :n] = -cN[:n] / S
                    F[n, n] = 1.0 / S
                self.tau[n], self.site[n], self.s[n] = tau, site, s_new
                self.order.append(n)
                self.n = n + 1
        else:
            if n == 0:
                rec.update(ratio=(0.0, 0.0), accept=False)
                self.trace.append(rec)
                return rec
            i = min(int(u_idx * n), n - 1)
            p = self.order[i]
            f = n / self.m.K
            r = (self.N[0][p, p], self.N[1][p, p])
            rec["ratio"] = r
            acc = u < min(1.0, abs(f * r[0] * r[1]))
            if acc:
                last = n - 1
                for spin in (0, 1):
                    F = self.N[spin]
                    col = F[:, p].copy()
                    row = F[p, :].copy()
                    blas.dger(-1.0 / col[p], col, row, a=F, overwrite_a=1)
                    if p != last:          # the last slot moves into the freed one
                        F[p, :n] = F[last, :n]
                        F[:n, p] = F[:n, last]
                        F[p, p] = F[last, last]
                    F[last, :n] = 0.0
                    F[:n, last] = 0.0
                del self.order[i]
                if p != last:
                    self.tau[p], self.site[p], self.s[p] = self.tau[last], self.site[last], self.s[last]
                    self.order[self.order.index(last)] = p
                self.n = last
        rec["accept"] = bool(acc)
        self.trace.append(rec)
        return rec


class Submatrix(_Chain):
    """Submatrix updates (Secs. III-IV): k_max proposals per block against a grown
    Gamma^{-1}, then one Woodbury update of N with the s=0 rows removed."""

    def __init__(self, model, draws, k_max, p_insert=0.5):
        super().__init__(model, draws, p_insert)
        self.k_max = int(k_max)

    def block(self):
        m_ = self.m
        n = len(self.tau)
        props = [self.proposal(self.t + j) for j in range(self.k_max)]
        ins = [j for j, p in enumerate(props) if p[0] == INSERT]
        k_ins = len(ins)
        # pre-insertion: s = 0 vertices in slots n .. n + k_ins (Sec. IV A)
        tau = np.concatenate([self.tau, [props[j][2] for j in ins]])
        site = np.concatenate([self.site, np.array([props[j][3] for j in ins], np.int64)])
        s0 = np.concatenate([self.s, np.zeros(k_ins, np.int64)])
        m = n + k_ins
        slot_of = {j: n + a for a, j in enumerate(ins)}
        Next, Gcol, ev0 = [], [], []
        for spin in (0, 1):
            e = m_.ev(spin, s0)
            ev0.append(e)
            Ne = np.zeros((m, m))
            Ne[:n, :n] = self.N[spin]
            if k_ins:
                C = m_.g0(spin, tau[n:, None], site[n:, None], tau[None, :n], site[None, :n]) \
                    * (e[:n] - 1.0)[None, :]
                B = m_.g0(spin, tau[:, None], site[:, None], tau[None, n:], site[None, n:])
                Ne[n:, :n] = C @ self.N[spin]          # R~ = C N
                Ne[n:, n:] = np.eye(k_ins)
                Gc = Ne @ B                            # G = N_ext G0 for the new columns
            else:
                Gc = np.zeros((m, 0))
            Next.append(Ne)
            Gcol.append(Gc)

        def gcol(spin, rows, j):
            """Interacting G^0[rows, j] of the block start (Eq. NfromG for an old column)."""
            rows = np.asarray(rows, np.int64)
            if j < n:
                e = ev0[spin][j]
                return (Next[spin][rows, j] * e - (rows == j)) / (e - 1.0)
            return Gcol[spin][rows, j - n]

        def grow(spin, i, cols):
            """G^0[i, cols] (old columns by Eq. NfromG, new ones from the products)."""
            cols = np.asarray(cols, np.int64)
            out = np.empty(len(cols))
            old = cols < n
            co = cols[old]
            e = ev0[spin][co]
            out[old] = (Next[spin][i, co] * e - (co == i)) / (e - 1.0)
            out[~old] = Gcol[spin][i, cols[~old] - n]
            return out

        s = s0.copy()
        P, lam = [], []                  # touched slots, their cumulative lambda per spin
        Gi = [np.zeros((0, 0)), np.zeros((0, 0))]
        n_cur = n
        alive = [i for i in range(n)]    # interacting slots in birth order
        for j, (move, u, _tau, _site, s_new, u_idx) in enumerate(props):
            t = self.t + j
            rec = {"t": t, "move": move, "n": n_cur}
            if move == INSERT:
                p = slot_of[j]
                f = m_.K / (n_cur + 1)
            else:
                if n_cur == 0:
                    rec.update(ratio=(0.0, 0.0), accept=False)
                    self.trace.append(rec)
                    continue
                p = alive[min(int(u_idx * n_cur), n_cur - 1)]
                s_new = 0
                f = n_cur / m_.K
            lam_new = [float(m_.ev(spin, s_new - s0[p])) - 1.0 for spin in (0, 1)]
            q = P.index(p) if p in P else -1
            ratios, upd = [], []
            for spin in (0, 1):
                ln = lam_new[spin]
                if q < 0:
                    sv = gcol(spin, P, p)
                    wv = grow(spin, p, P)
                    y = Gi[spin] @ sv if P else sv
                    gpp = gcol(spin, [p], p)[0]
                    beta = gpp - (1.0 + ln) / ln - (wv @ y if P else 0.0)
                    ratios.append(-ln * beta)
                    upd.append(("grow", beta, y, wv))
                else:
                    lo = lam[q][spin]
                    gqq = Gi[spin][q, q]
                    if ln != 0.0:
                        delta = 1.0 / lo - 1.0 / ln
                        ratios.append((ln / lo) * (1.0 + delta * gqq))
                        upd.append(("diag", delta))
                    else:
                        ratios.append(-gqq / lo)
                        upd.append(("drop",))
            R = f * ratios[0] * ratios[1]
            rec["ratio"] = tuple(ratios)
            acc = u < min(1.0, abs(R))
            rec["accept"] = bool(acc)
            self.trace.append(rec)
            if not acc:
                continue
            for spin in (0, 1):
                G = Gi[spin]
                kind = upd[spin][0]
                if kind == "grow":
                    _, beta, y, wv = upd[spin]
                    z = wv @ G if P else wv
                    jn = len(P)
                    Gn = np.empty((jn + 1, jn + 1))
                    Gn[:jn, :jn] = G + np.outer(y, z) / beta
                    Gn[:jn, jn] = -y / beta
                    Gn[jn, :jn] = -z / beta
                    Gn[jn, jn] = 1.0 / beta
                    Gi[spin] = Gn
                elif kind == "diag":
                    delta = upd[spin][1]
                    Gi[spin] = G - np.outer(G[:, q], G[q, :]) * (delta / (1.0 + delta * G[q, q]))
                else:
                    G = G - np.outer(G[:, q], G[q, :]) / G[q, q]
                    keep = [r for r in range(len(P)) if r != q]
                    Gi[spin] = G[np.ix_(keep, keep)]
            if q < 0:
                P.append(p)
                lam.append(lam_new)
            elif lam_new[0] != 0.0:
                lam[q] = lam_new
            else:
                del P[q]
                del lam[q]
            s[p] = s_new
            if move == INSERT:
                alive.append(p)
                n_cur += 1
            else:
                alive.remove(p)
                n_cur -= 1
        # flush (Eq. Nshermanmorrison, D^{-1} folded): N' = N_SS - (G - 1)_{S,P} Gamma^{-1} N_{P,S}
        S = np.array(sorted(alive), dtype=np.int64)
        for spin in (0, 1):
            Ne = Next[spin]
            if P:
                GSP = np.stack([gcol(spin, S, pp) - (S == pp) for pp in P], axis=1)
                Y = GSP @ Gi[spin]
                self.N[spin] = Ne[np.ix_(S, S)] - Y @ Ne[np.ix_(P, S)]
            else:
                self.N[spin] = Ne[np.ix_(S, S)]
        self.tau, self.site, self.s = tau[S], site[S], s[S]
        self.t += self.k_max


def time_algorithms(chain_input, n0, ks, n_props, seed=7):
    """Proposals per second of the rank-one and submatrix algorithms from the same
    seeded configuration of order n0 (one thread).  Returns rows per algorithm."""
    ch = chain_input
    model = Model(ch.table, ch.dx_class, ch.beta, ch.U, ch.K)
    rng = np.random.default_rng(seed)
    tau0 = rng.uniform(0.0, ch.beta, n0)
    site0 = rng.integers(0, ch.n_c, n0)
    s0 = rng.choice([-1, 1], n0)
    rows = []
    algos = [("rank_one", 1)] + [("submatrix", k) for k in ks]
    for name, k in algos:
        c = RankOne(model, numpy_draws(seed)) if name == "rank_one" else \
            Submatrix(model, numpy_draws(seed), k)
        c.set_config(tau0, site0, s0, 0)
        done, acc = 0, 0
        t0 = time.perf_counter()
        while done < n_props:
            if name == "rank_one":
                acc += int(c.step()["accept"])
                done += 1
            else:
                before = len(c.trace)
                c.block()
                acc += sum(int(r["accept"]) for r in c.trace[before:])
                done += k
        dt = time.perf_counter() - t0
        n_end = c.n if name == "rank_one" else len(c.tau)
        rows.append({"algorithm": name, "k_max": k, "order_n0": n0, "order_end": n_end,
                     "proposals": done, "seconds": dt, "proposals_per_s": done / dt,
                     "accepted_per_s": acc / dt})
    return rows
