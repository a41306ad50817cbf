"""A second, vectorised numpy Philox4x32-10 written for the tests.

Written from the published round function (Salmon et al., SC'11): per round
two 32x32 -> 64-bit products of counter words 0 and 2 with 0xD2511F53 and
0xCD9E8D57, the output words being (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
and the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.  Used to
re-derive photon launch positions in brute-force tests, and cross-checked
against the C oracle and the published known-answer vectors.
"""
from __future__ import annotations

import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    c = [np.asarray(x, dtype=np.uint64) & MASK32 for x in (c0, c1, c2, c3)]
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ np.uint64(k0)) & MASK32, p1 & MASK32,
             ((p0 >> np.uint64(32)) ^ c[3] ^ np.uint64(k1)) & MASK32, p0 & MASK32]
    return [x.astype(np.uint32) for x in c]


def uniform(r):
    r = np.asarray(r, dtype=np.uint32)
    return ((r >> np.uint32(9)).astype(np.float64) * 2.0 + 1.0) * 2.0 ** -24


def event_words(pids, j: int, seed: int):
    """Words of event j for photon ids ``pids`` under a 64-bit seed."""
    pids = np.asarray(pids, dtype=np.uint64)
    return philox4x32_10(np.full(pids.shape, j, dtype=np.uint64), np.zeros(pids.shape, np.uint64),
                         pids & MASK32, pids >> np.uint64(32), seed & 0xFFFFFFFF, seed >> 32)
