"""Exact diagonalisation of a small Anderson impurity: the pin of the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Two independent routes to numbers the CT-AUX oracle must reproduce:

1. Interacting impurity (Eq. Ham with a discrete bath): build the many-body
   Hamiltonian of impurity + bath levels, both spins, by Jordan-Wigner, and
   diagonalise it.  Gives G(tau) = -<T d(tau) d^dagger(0)>, the density and the
   double occupancy <n_up n_down>.

2. One spin species at U = 0 with an explicit time-ordered product of the
   auxiliary-field exponentials: Tr[T prod_i e^{v_i n(tau_i)} e^{-beta H0}]/Z0
   and the Green's function in the presence of those exponentials.  This pins
   the weight formula det N^{-1} (Eq. Zn_div_Z0, Eq. Nmatrix) and the G
   estimator configuration by configuration, with operators instead of
   determinants.
"""
from __future__ import annotations

import numpy as np

from workloads import g0tables


def fermion_ops(n_modes):
    """Dense annihilation operators c_i on the 2^n_modes Fock space (Jordan-Wigner)."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])   # |1> -> |0>
    z = np.diag([1.0, -1.0])
    eye = np.eye(2)
    ops = []
    for i in range(n_modes):
        m = np.array([[1.0]])
        for j in range(n_modes):
            m = np.kron(m, z if j < i else (a if j == i else eye))
        ops.append(m)
    return ops


def _thermal_trace(E, V, beta, ops_times):
    """Tr[e^{-(beta-t1) H} O1 e^{-(t1-t2) H} O2 ... Ok e^{-tk H}] / Z in the eigenbasis.

    ops_times: list of (t, O) sorted with t descending; O in the original basis.
    """
    e0 = E.min()
    Es = E - e0
    prev = beta
    M = np.eye(len(E))
    for t, O in ops_times:
        M = M @ np.diag(np.exp(-(prev - t) * Es)) @ (V.T @ O @ V)
        prev = t
    M = M @ np.diag(np.exp(-prev * Es))
    Z = np.exp(-beta * Es).sum()
    return np.trace(M) / Z


class AndersonED:
    """Impurity (mode 0) + bath levels, both spins; spin-up modes first."""

    def __init__(self, beta, U, eps_bath=(-1.0, 0.0, 1.0), v_bath=(0.5, 0.5, 0.5), eps_imp=0.0):
        self.beta = float(beta)
        nb = len(eps_bath)
        no = nb + 1
        self.no = no
        c = fermion_ops(2 * no)
        self.c = c
        h1 = g0tables.aim_single_particle_h(eps_bath, v_bath, eps_imp)
        H = np.zeros_like(c[0])
        for sp in range(2):
            for i in range(no):
                for j in range(no):
                    if h1[i, j] != 0.0:
                        H += h1[i, j] * c[sp * no + i].T @ c[sp * no + j]
        nu = c[0].T @ c[0]
        nd = c[no].T @ c[no]
        # V = U [n_up n_down - (n_up + n_down)/2]  (Eq. Ham)
        H += U * (nu @ nd - 0.5 * (nu + nd))
        self.E, self.V = np.linalg.eigh(H)
        self.nu, self.nd = nu, nd

    def G(self, taus, spin=0):
        d = self.c[spin * self.no]
        return np.array([-_thermal_trace(self.E, self.V, self.beta, [(t, d), (0.0, d.T)])
                         for t in np.atleast_1d(taus)])

    def G_matsubara(self, w, spin=0):
        """G(iw) = int_0^beta e^{iw tau} G(tau) dtau by the Lehmann sum
        (1/Z) sum_nm |<n|d|m>|^2 (e^{-beta E_n} + e^{-beta E_m}) / (iw + E_n - E_m)."""
        A = self.V.T @ self.c[spin * self.no] @ self.V
        Es = self.E - self.E.min()
        bw = np.exp(-self.beta * Es)
        num = (A ** 2) * (bw[:, None] + bw[None, :])
        den = Es[:, None] - Es[None, :]
        w = np.atleast_1d(np.asarray(w, dtype=np.float64))
        return np.array([np.sum(num / (1j * wi + den)) for wi in w]) / bw.sum()

    def double_occupancy(self):
        return _thermal_trace(self.E, self.V, self.beta, [(0.0, self.nu @ self.nd)])

    def density(self, spin=0):
        return _thermal_trace(self.E, self.V, self.beta, [(0.0, self.nu if spin == 0 else self.nd)])


class SingleSpinFreeED:
    """Non-interacting impurity + bath for ONE spin species (2^(nb+1) states)."""

    def __init__(self, beta, eps_bath=(-1.0, 0.0, 1.0), v_bath=(0.5, 0.5, 0.5), eps_imp=0.0):
        self.beta = float(beta)
        h1 = g0tables.aim_single_particle_h(eps_bath, v_bath, eps_imp)
        no = h1.shape[0]
        c = fermion_ops(no)
        H = np.zeros_like(c[0])
        for i in range(no):
            for j in range(no):
                if h1[i, j] != 0.0:
                    H += h1[i, j] * c[i].T @ c[j]
        self.E, self.V = np.linalg.eigh(H)
        self.d = c[0]
        self.n = c[0].T @ c[0]
        self.h1 = h1

    def g0_matsubara(self, w):
        """G0(iw) = sum_k |U_0k|^2 / (iw - E_k) from the single-particle levels."""
        E, U = np.linalg.eigh(self.h1)
        wt = U[0, :] ** 2
        w = np.atleast_1d(np.asarray(w, dtype=np.float64))
        return (wt[None, :] / (1j * w[:, None] - E[None, :])).sum(axis=1)

    def _exp_n(self, v):
        # e^{v n} = 1 + (e^v - 1) n
        return np.eye(len(self.E)) + (np.exp(v) - 1.0) * self.n

    def weight(self, taus, vs):
        """<T prod_i e^{v_i n(tau_i)}>_0 (bosonic operators, no fermion sign)."""
        ops = sorted([(t, self._exp_n(v)) for t, v in zip(taus, vs)], key=lambda p: -p[0])
        return _thermal_trace(self.E, self.V, self.beta, ops)

    def green(self, tau_a, tau_b, taus, vs):
        """-<T d(tau_a) d^dagger(tau_b) prod_i e^{v_i n(tau_i)}> / <T prod_i e^{v_i n(tau_i)}>."""
        ops = [(t, self._exp_n(v)) for t, v in zip(taus, vs)]
        ops.append((tau_a, self.d))
        ops.append((tau_b, self.d.T))
        ops = sorted(ops, key=lambda p: -p[0])
        sign = -1.0 if tau_b > tau_a else 1.0   # fermionic reordering of d, d^dagger
        num = sign * _thermal_trace(self.E, self.V, self.beta, ops)
        return -num / self.weight(taus, vs)
