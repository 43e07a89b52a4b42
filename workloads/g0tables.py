"""Bare (non-interacting) Green's function tables: the physics input of CT-AUX.

The solver consumes a tabulated bath Green's function G0_sigma(dx, tau) on a
uniform grid tau_j = j*beta/(n_tau-1), j = 0..n_tau-1 (both ends included), one
row per displacement class dx of the cluster.  The sign convention is
G0(tau) = -<T d(tau) d^dagger(0)>, negative on (0, beta); the table holds the
limits G0(0+) at j=0 and G0(beta-) at j=n_tau-1.

This module only builds inputs.  It holds none of the submatrix-update
arithmetic (no interpolation, no N matrices, no determinants); the solver and
the oracle each read the tables with their own code.

Models (paper Sec. II for the Anderson model, Eq. Ham; Sec. V for the DCA
clusters of the 3D Hubbard model):
  * semicircular density of states, half-bandwidth D (single-site impurity);
  * DCA coarse-grained cluster G0 of the simple-cubic / square lattice
    (non-interacting lattice, coarse-grained over the cluster patches);
  * a 1-site Anderson impurity with a few discrete bath levels (exactly
    solvable by diagonalisation; used to pin the oracle).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def fermion_g(xi, tau, beta):
    """-exp(-xi*tau)/(1+exp(-beta*xi)) for 0 <= tau <= beta, overflow-safe.

    xi and tau broadcast against each other.  For xi < 0 the equivalent form
    -exp(xi*(beta-tau))/(1+exp(beta*xi)) is used so no exponent is positive.
    """
    xi = np.asarray(xi, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    xi_b, tau_b = np.broadcast_arrays(xi, tau)
    out = np.empty(xi_b.shape, dtype=np.float64)
    pos = xi_b >= 0.0
    xp, tp = xi_b[pos], tau_b[pos]
    out[pos] = -np.exp(-xp * tp) / (1.0 + np.exp(-beta * xp))
    xn, tn = xi_b[~pos], tau_b[~pos]
    out[~pos] = -np.exp(xn * (beta - tn)) / (1.0 + np.exp(beta * xn))
    return out


def tau_grid(beta, n_tau):
    return np.linspace(0.0, beta, n_tau)


# --------------------------------------------------------------------------
# semicircle
# --------------------------------------------------------------------------
def semicircle_g0(beta, n_tau, D=2.0, mu=0.0, n_quad=4000):
    """G0(tau) of a level coupled to a semicircular DOS rho(e)=2/(pi D^2) sqrt(D^2-e^2).

    Gauss-Chebyshev quadrature of the second kind: with e = D x,
    int rho(e) f(e) de = (2/pi) int_{-1}^{1} sqrt(1-x^2) f(D x) dx
                       ~ (2/pi) sum_i w_i f(D x_i),
    x_i = cos(i pi/(n+1)), w_i = pi/(n+1) sin^2(i pi/(n+1)).
    Returns an array of shape [n_tau].
    """
    i = np.arange(1, n_quad + 1)
    theta = i * math.pi / (n_quad + 1)
    x = np.cos(theta)
    w = (math.pi / (n_quad + 1)) * np.sin(theta) ** 2 * (2.0 / math.pi)
    taus = tau_grid(beta, n_tau)
    out = np.empty(n_tau)
    chunk = 512
    for s in range(0, n_tau, chunk):
        t = taus[s:s + chunk, None]
        out[s:s + chunk] = fermion_g(D * x[None, :] - mu, t, beta) @ w
    return out


# --------------------------------------------------------------------------
# DCA clusters
# --------------------------------------------------------------------------
class Cluster:
    """A periodic cluster of the hypercubic lattice given by superlattice vectors.

    Attributes:
      A      integer superlattice vectors as rows, shape [d, d]
      sites  integer site coordinates inside the cluster cell, shape [n_c, d]
      K      cluster momenta, shape [n_c, d]
      dx_class[i][j] = index of the site equal to (r_i - r_j) mod superlattice
    """

    def __init__(self, A):
        A = np.array(A, dtype=np.int64)
        d = A.shape[0]
        self.A = A
        self.d = d
        n_c = int(round(abs(np.linalg.det(A))))
        self.n_c = n_c
        At_inv = np.linalg.inv(A.T.astype(np.float64))
        span = int(np.abs(A).sum(axis=0).max()) + 1
        sites = []
        for r in itertools.product(range(-span, span + 1), repeat=d):
            f = At_inv @ np.array(r, dtype=np.float64)
            if np.all(f >= -1e-9) and np.all(f < 1.0 - 1e-9):
                sites.append(r)
        sites = sorted(sites, key=lambda r: (sum(abs(v) for v in r), r))
        # put the origin first
        assert tuple([0] * d) in sites
        sites.remove(tuple([0] * d))
        sites.insert(0, tuple([0] * d))
        self.sites = np.array(sites, dtype=np.int64)
        assert len(self.sites) == n_c, (len(self.sites), n_c)
        self._At_inv = At_inv
        index = {tuple(r): i for i, r in enumerate(self.sites)}
        self.dx_class = np.empty((n_c, n_c), dtype=np.int32)
        for i in range(n_c):
            for j in range(n_c):
                self.dx_class[i, j] = index[self.reduce(self.sites[i] - self.sites[j])]
        # reciprocal superlattice b = 2 pi A^{-T} (rows).  Cluster momenta
        # K = 2 pi phi with phi = m A^{-T}; n_c * phi is an integer vector, so the
        # momenta are enumerated and reduced modulo 2 pi in exact integers.
        self.B = 2.0 * math.pi * np.linalg.inv(A.astype(np.float64)).T
        adjT = np.round(np.linalg.inv(A.astype(np.float64)).T * n_c).astype(np.int64)
        ks = {}
        for m in itertools.product(range(n_c), repeat=d):
            num = (np.array(m, dtype=np.int64) @ adjT) % n_c           # n_c * phi mod n_c
            num = np.where(num >= (n_c + 1) // 2, num - n_c, num)      # to [-n_c/2, n_c/2)
            key = tuple(int(v) for v in num)
            if key not in ks:
                ks[key] = 2.0 * math.pi * num.astype(np.float64) / n_c
            if len(ks) == n_c:
                break
        self.K = np.array([ks[k] for k in sorted(ks)])
        assert len(self.K) == n_c
        # exp(i K . a) = 1 for every superlattice vector a
        assert np.allclose(np.exp(1j * (self.K @ A.T.astype(np.float64))), 1.0)

    def reduce(self, r):
        f = self._At_inv @ np.asarray(r, dtype=np.float64)
        n = np.floor(f + 1e-9)
        red = np.asarray(r, dtype=np.float64) - self.A.T.astype(np.float64) @ n
        return tuple(int(round(v)) for v in red)


def dispersion(k, t=1.0, tp=0.0):
    """Hypercubic nearest-neighbour band (plus 2D next-nearest t' when d=2)."""
    k = np.atleast_2d(k)
    e = -2.0 * t * np.cos(k).sum(axis=1)
    if k.shape[1] == 2 and tp != 0.0:
        e = e - 4.0 * tp * np.cos(k[:, 0]) * np.cos(k[:, 1])
    return e


def _patch_offsets(cl, n_grid):
    f = (np.arange(n_grid) + 0.5) / n_grid - 0.5
    grid = np.array(list(itertools.product(f, repeat=cl.d)))
    return grid @ cl.B  # [n_grid^d, d]


def cluster_density(cl, beta, mu, t=1.0, tp=0.0, n_grid=16):
    """Non-interacting density per site and spin of the lattice (Fermi average)."""
    kt = _patch_offsets(cl, n_grid)
    tot = 0.0
    for K in cl.K:
        xi = dispersion(K[None, :] + kt, t, tp) - mu
        tot += np.mean(0.5 * (1.0 - np.tanh(0.5 * beta * xi)))
    return tot / cl.n_c


def mu_for_density(cl, beta, density_per_site, t=1.0, tp=0.0, n_grid=16):
    """Bisect mu so the non-interacting lattice holds the given total density."""
    target = 0.5 * density_per_site
    lo, hi = -12.0 * abs(t) - 8, 12.0 * abs(t) + 8
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if cluster_density(cl, beta, mid, t, tp, n_grid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def cluster_g0(cl, beta, n_tau, mu=0.0, t=1.0, tp=0.0, n_grid=12, k_chunk=2048):
    """Coarse-grained cluster G0(dx, tau), shape [n_c(classes), n_tau].

    G0(K, tau) = (1/N_p) sum_{k~ in patch} g(eps(K+k~) - mu, tau) with the patch
    a fundamental cell of the reciprocal superlattice centred on K (the patches
    of all K tile the Brillouin zone once), then
    G0(dx, tau) = (1/N_c) sum_K exp(i K.dx) G0(K, tau).
    Row c of the result is the displacement of cluster site c.
    """
    taus = tau_grid(beta, n_tau)
    kt = _patch_offsets(cl, n_grid)
    gK = np.zeros((cl.n_c, n_tau))
    for iK, K in enumerate(cl.K):
        xi = dispersion(K[None, :] + kt, t, tp) - mu
        acc = np.zeros(n_tau)
        for s in range(0, len(xi), k_chunk):
            acc += fermion_g(xi[s:s + k_chunk, None], taus[None, :], beta).sum(axis=0)
        gK[iK] = acc / len(xi)
    phase = np.exp(1j * (cl.sites.astype(np.float64) @ cl.K.T))  # [n_c sites, n_c K]
    gx = (phase @ gK) / cl.n_c
    assert np.max(np.abs(gx.imag)) < 1e-10 * max(1.0, np.max(np.abs(gx.real)))
    return np.ascontiguousarray(gx.real)


# --------------------------------------------------------------------------
# Anderson impurity with discrete bath (exactly solvable)
# --------------------------------------------------------------------------
def aim_single_particle_h(eps_bath, v_bath, eps_imp=0.0):
    nb = len(eps_bath)
    h = np.zeros((nb + 1, nb + 1))
    h[0, 0] = eps_imp
    for p in range(nb):
        h[0, p + 1] = h[p + 1, 0] = v_bath[p]
        h[p + 1, p + 1] = eps_bath[p]
    return h


def aim_g0(beta, n_tau, eps_bath=(-1.0, 0.0, 1.0), v_bath=(0.5, 0.5, 0.5), eps_imp=0.0):
    """Impurity G0(tau) of the non-interacting Anderson model, shape [n_tau].

    eps_imp is the impurity level of H0 after the U/2 shift of Eq. Ham
    (eps_imp = 0 is the particle-hole symmetric point).
    """
    h = aim_single_particle_h(eps_bath, v_bath, eps_imp)
    E, U = np.linalg.eigh(h)
    w = U[0, :] ** 2
    taus = tau_grid(beta, n_tau)
    return fermion_g(E[None, :], taus[:, None], beta) @ w


def tables_for_spins(g0_rows):
    """Stack one spin's [n_classes, n_tau] table into the paramagnetic [2, ...] form."""
    g = np.asarray(g0_rows, dtype=np.float64)
    if g.ndim == 1:
        g = g[None, :]
    return np.ascontiguousarray(np.stack([g, g]))
