"""Counter-based random numbers (oracle; test infrastructure).

Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011), written here from its published definition: a
128-bit counter (four 32-bit words) is mixed with a 64-bit key (two words)
by ten rounds.  One round multiplies counter words 0 and 2 by two fixed odd
32-bit constants, keeps each 64-bit product's high and low halves, and
forms the new counter as

    (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0)),

after which the key is advanced by two fixed "Weyl" increments (the first
round uses the key as given).  The CUDA path implements the same published
generator on its own; the two share no code.

Uses here: the seeded He initialisation of the warm-start network, and the
re-loading of absorbed ions as thermal ions in the bulk (ion recycling of
Sec. III-A and III-C), both keyed so that every draw is a pure function of
(seed, step, particle id) and independent of thread or particle order.

Pinned by the published known-answer vectors of Philox4x32-10
(tests/golden/philox4x32_10_kat.txt).
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """ctr: uint array [..., 4], key: uint array [..., 2] (broadcast);
    returns the four output words as uint64 arrays [..., 4] < 2^32."""
    c = np.asarray(ctr, dtype=np.uint64) & np.uint64(MASK)
    k = np.asarray(key, dtype=np.uint64) & np.uint64(MASK)
    c0, c1, c2, c3 = (c[..., q].copy() for q in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    m0, m1 = np.uint64(M0), np.uint64(M1)
    mask = np.uint64(MASK)
    s32 = np.uint64(32)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(W0)) & mask
            k1 = (k1 + np.uint64(W1)) & mask
        p0 = m0 * c0          # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def seed_key(seed):
    """The 64-bit seed as the two key words (low word first)."""
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([s & MASK, s >> 32], dtype=np.uint64)


def unit24(word):
    """The top 24 bits of a 32-bit word as a float in [0, 1) (exact in FP32)."""
    return (np.asarray(word, np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def unit24_open(word):
    """As unit24 but in (0, 1]: the logarithm of Box-Muller needs u > 0."""
    return ((np.asarray(word, np.uint64) >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24


def below(word, n):
    """floor(word * n / 2^32): a uniform integer in [0, n) from a 32-bit word."""
    return ((np.asarray(word, np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def box_muller(u1, u2):
    """Two independent standard normals from u1 in (0, 1], u2 in [0, 1)
    (Box and Muller, 1958): r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2)."""
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)
