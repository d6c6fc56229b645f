"""Philox4x32-10 counter-based generator (oracle side).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the timed
CPU baseline; the CUDA path never imports it.

Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel
Random Numbers: As Easy as 1, 2, 3", SC'11): ten rounds of

    (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),

M0 = 0xD2511F53, M1 = 0xCD9E8D57, with the key (k0, k1) advanced by the Weyl
constants (0x9E3779B9, 0xBB67AE85) after every round. Vectorised over numpy
uint32 arrays; products are formed in uint64.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four output words (uint32 arrays) for counters (c0..c3) and key (k0, k1)."""
    c = [np.asarray(x, dtype=np.uint32).copy() for x in np.broadcast_arrays(c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint32).copy()
    k1 = np.asarray(k1, dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = M0 * c[0].astype(np.uint64)
            p1 = M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK32).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = k0 + W0
            k1 = k1 + W1
    return c


def uniform_index(u32, d):
    """Neighbour index in [0, d) from one 32-bit word: floor(u * d / 2^32)
    (Lemire's multiply-shift; bias at most d / 2^32)."""
    return ((np.asarray(u32, dtype=np.uint64) * np.asarray(d, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)
