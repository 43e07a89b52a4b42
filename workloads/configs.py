"""The benchmark workloads as seeded, synthetic inputs.

Each workload is a list of chains; a chain is the full input of one CT-AUX
Markov chain: the G0 table [2][n_classes][n_tau], the displacement-class map
[n_c][n_c], (beta, U, K), the submatrix size k_max, a capacity for the
expansion order, and the Philox seed / chain id.  Nothing here computes any
part of the submatrix update.

Workloads (the paper's model systems: Sec. II Anderson impurity, Sec. V 3D
Hubbard DCA clusters; sizes chosen to span the paper's range of expansion
orders 20..8000, Sec. V A):
  aim1     N_c=1 semicircular DOS (D=2), beta=10, U=4, K=1, 10^4 tau points, k=8
  cube8    N_c=8 2x2x2 simple-cubic cluster, beta=5, U=8, 4096 tau points, k=16..64
  sq36     N_c=36 6x6 square cluster, density 0.9, beta=8, U=6, k=64..128
  batch    many chains, N_c in {4,8,16}, beta in U[2,10], U in U[4,10]
  cube100  N_c=100 3D cluster, beta=4, U=8, k=128..256
  aim_ed   1-site Anderson impurity with 3 bath levels (exact diagonalisation pin)
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

from . import g0tables as g0t

SUPERLATTICES = {
    1: [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
    4: [[1, 1, 0], [1, -1, 0], [0, 0, 2]],
    8: [[2, 0, 0], [0, 2, 0], [0, 0, 2]],
    16: [[2, 2, 0], [2, -2, 0], [0, 0, 2]],
    100: [[5, 5, 0], [5, -5, 0], [0, 0, 2]],
}


@dataclasses.dataclass
class ChainInput:
    name: str
    n_c: int
    table: np.ndarray        # [2, n_classes, n_tau] float64
    dx_class: np.ndarray     # [n_c, n_c] int32
    beta: float
    U: float
    K: float
    k_max: int
    capacity: int
    seed: int = 0
    chain_id: int = 0

    @property
    def n_classes(self):
        return self.table.shape[1]

    @property
    def n_tau(self):
        return self.table.shape[2]


@functools.lru_cache(maxsize=None)
def cluster(n_c):
    if n_c == 36:
        return g0t.Cluster([[6, 0], [0, 6]])
    return g0t.Cluster(SUPERLATTICES[n_c])


@functools.lru_cache(maxsize=None)
def _cluster_table(n_c, beta, n_tau, density, n_grid):
    cl = cluster(n_c)
    mu = 0.0 if density == 1.0 else g0t.mu_for_density(cl, beta, density, n_grid=n_grid)
    return g0t.cluster_g0(cl, beta, n_tau, mu=mu, n_grid=n_grid)


def cluster_chain(name, n_c, beta, U, K, k_max, capacity, n_tau=4096, density=1.0,
                  seed=0, chain_id=0, n_grid=None):
    cl = cluster(n_c)
    if n_grid is None:
        n_grid = {1: 64, 4: 24, 8: 12, 16: 10, 36: 12, 100: 6}[n_c]
    rows = _cluster_table(n_c, float(beta), n_tau, float(density), n_grid)
    return ChainInput(name, n_c, g0t.tables_for_spins(rows), cl.dx_class.copy(), float(beta),
                      float(U), float(K), int(k_max), int(capacity), int(seed), int(chain_id))


@functools.lru_cache(maxsize=None)
def _semicircle(beta, n_tau):
    return g0t.semicircle_g0(beta, n_tau)


def aim1(K=1.0, k_max=8, capacity=256, n_tau=10000, seed=0, beta=10.0, U=4.0):
    tab = g0t.tables_for_spins(_semicircle(float(beta), n_tau))
    return ChainInput("aim1", 1, tab, np.zeros((1, 1), np.int32), beta, U, K, k_max, capacity,
                      seed, 0)


def aim_ed(beta=5.0, U=4.0, K=1.0, k_max=8, capacity=128, n_tau=4001, seed=0,
           eps_bath=(-1.0, 0.0, 1.0), v_bath=(0.5, 0.5, 0.5)):
    tab = g0t.tables_for_spins(g0t.aim_g0(beta, n_tau, eps_bath, v_bath))
    return ChainInput("aim_ed", 1, tab, np.zeros((1, 1), np.int32), beta, U, K, k_max, capacity,
                      seed, 0)


def cube8(K=1.0, k_max=64, capacity=None, seed=0):
    if capacity is None:
        capacity = 256 if K <= 1.0 else 1024
    return cluster_chain("cube8", 8, 5.0, 8.0, K, k_max, capacity, n_tau=4096, seed=seed)


def sq36(K=1.0, k_max=128, capacity=3072, seed=0):
    return cluster_chain("sq36", 36, 8.0, 6.0, K, k_max, capacity, n_tau=4096, density=0.9,
                         seed=seed)


def cube100(K=1.0, k_max=256, capacity=9216, seed=0, chain_id=0):
    return cluster_chain("cube100", 100, 4.0, 8.0, K, k_max, capacity, n_tau=4096,
                         seed=seed, chain_id=chain_id)


def batch(n_chains=512, seed=12345, k_max=32, K=None, capacity=None, n_tau=1024):
    """Independent chains of uneven size: N_c in {4,8,16}, beta~U[2,10], U~U[4,10].

    Parameters are drawn from a numpy Generator with a fixed seed; beta is
    rounded to a multiple of 0.5 so that chains share G0 tables (17 x 3
    tables instead of one per chain); the Philox seed of chain i is i (the
    chain id goes into the counter as well).  K=None picks the expansion
    constant per chain as K = 0.3 beta U N_c + 30, which puts the orders at
    n ~ K + 0.4 beta U N_c ~ 50..1200 (the batch's named range) and keeps
    cosh(gamma) = 1 + beta U N_c / (2K) below ~2.7.
    """
    rng = np.random.default_rng(seed)
    chains = []
    for i in range(n_chains):
        n_c = int(rng.choice([4, 8, 16]))
        beta = float(np.round(rng.uniform(2.0, 10.0) * 2.0) / 2.0)
        U = float(np.round(rng.uniform(4.0, 10.0), 3))
        Ki = float(K) if K is not None else round(0.3 * beta * U * n_c + 30.0, 3)
        cap = capacity
        if cap is None:
            # expected order K + beta U N_c / 2 (no double occupancy) plus headroom
            cap = int(math.ceil((Ki + 0.5 * beta * U * n_c) * 1.25 / 32.0)) * 32 + 64
        chains.append(cluster_chain("batch", n_c, beta, U, Ki, k_max, cap, n_tau=n_tau,
                                    seed=i, chain_id=i))
    return chains


def expected_order(beta, U, n_c, K, double_occ, density=1.0):
    """<n> = K - beta <V> = K + beta U N_c (density/2 - d) (follows from Eq. decoupledZ)."""
    return K + beta * U * n_c * (0.5 * density - double_occ)


def synthetic_configuration(ch, n, seed=0, t0=None):
    """A seeded configuration of n interacting vertices for checkpoint starts.

    tau ~ U[0, beta), site ~ U{0..N_c-1}, s = +-1 with equal probability, birth
    stamps 0..n-1 (canonical order), next proposal counter t0 (default
    2^20 + n).  Not an equilibrium sample: a valid Markov-chain state of the
    requested size, used as the common starting point of the CUDA path and the
    oracle.
    """
    rng = np.random.default_rng(seed)
    return dict(tau=rng.uniform(0.0, ch.beta, n), site=rng.integers(0, ch.n_c, n).astype(np.int32),
                s=rng.choice(np.array([-1, 1], dtype=np.int32), n),
                birth=np.arange(n, dtype=np.int64),
                t=int(t0 if t0 is not None else (1 << 20) + n))
