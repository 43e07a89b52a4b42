"""Philox-4x32-10 counter-based generator, the oracle's own copy.

Written from the published description (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter and 2x32-bit
key; each of 10 rounds does two 32x32->64-bit multiplications with the
multipliers 0xD2511F53 and 0xCD9E8D57, xors the high halves with the other
counter words and the round key, and bumps the key by the Weyl constants
0x9E3779B9 and 0xBB67AE85.

The paper draws its proposals and Metropolis uniforms from an unspecified
generator; this counter-based one lets the oracle and the CUDA path replay the
same stream without sharing code (each implements it from the definition).

Counter layout used by the Markov chain: (t_lo, t_hi, chain, purpose), key =
(seed_lo, seed_hi).  A uniform in [0,1) takes 53 bits from two output words:
u = (w_a * 2^21 + (w_b >> 11)) * 2^-53.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)

# purposes (the 4th counter word); each call yields two uniforms
PURPOSE_MOVE_ACCEPT = 0   # (u_move, u_accept)
PURPOSE_TAU_SITE = 1      # (u_tau, u_site)
PURPOSE_SPIN_INDEX = 2    # (u_spin, u_index)


def philox4x32_10(ctr, key):
    """ctr: uint32-valued array [4, N] (or [4]); key: two ints. Returns uint32 [4, N]."""
    c = np.array(ctr, dtype=np.uint64).reshape(4, -1) & MASK
    x0, x1, x2, x3 = c[0].copy(), c[1].copy(), c[2].copy(), c[3].copy()
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = M0 * x0            # exact: both factors < 2^32
        p1 = M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        y0 = hi1 ^ x1 ^ np.uint64(k0)
        y2 = hi0 ^ x3 ^ np.uint64(k1)
        x0, x1, x2, x3 = y0, lo1, y2, lo0
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return np.stack([x0, x1, x2, x3]).astype(np.uint32)


def words_to_uniform(wa, wb):
    """53-bit uniform in [0, 1) from two 32-bit words (exact in float64)."""
    wa = np.asarray(wa, dtype=np.uint64)
    wb = np.asarray(wb, dtype=np.uint64)
    mant = (wa << np.uint64(21)) + (wb >> np.uint64(11))
    return mant.astype(np.float64) * (2.0 ** -53)


def uniforms(seed, chain, t, purpose):
    """The pair of uniforms for proposal index/indices t of a chain and a purpose.

    Returns (u_first, u_second) arrays matching t's shape.
    """
    t = np.asarray(t, dtype=np.uint64)
    flat = t.reshape(-1)
    n = flat.size
    ctr = np.empty((4, n), dtype=np.uint64)
    ctr[0] = flat & MASK
    ctr[1] = flat >> np.uint64(32)
    ctr[2] = np.uint64(chain & 0xFFFFFFFF)
    ctr[3] = np.uint64(purpose)
    seed = int(seed)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    ua = words_to_uniform(w[0], w[1]).reshape(t.shape)
    ub = words_to_uniform(w[2], w[3]).reshape(t.shape)
    return ua, ub
