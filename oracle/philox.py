"""Philox4x32-10 in plain numpy uint64 arithmetic (oracle; test infrastructure).

Definition followed: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3 (the Philox
S-box/P-box round on four 32-bit words with a two-word key).

One round maps counter (c0, c1, c2, c3) under key (k0, k1) to

    hi0:lo0 = M0 * c0          (full 64-bit product of two 32-bit words)
    hi1:lo1 = M1 * c2
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)

with M0 = 0xD2511F53 and M1 = 0xCD9E8D57. Between rounds the key is bumped
by the Weyl constants W0 = 0x9E3779B9, W1 = 0xBB67AE85 (mod 2^32). Ten rounds.

The paper draws its white noise from SPRNG 2.0 (Sec. 2.1); a counter-based
generator replaces it so that every cell's value depends only on
(seed, cell index). Bit compatibility with the paper's realizations is
impossible in any case.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
SHIFT32 = np.uint64(32)
ROUNDS = 10


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=ROUNDS):
    """Philox4x32-R on arrays (broadcast) of 32-bit words held in uint64.

    Returns four uint64 arrays, each holding a 32-bit output word.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3, k0, k1 = (a.copy() for a in (c0, c1, c2, c3, k0, k1))
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0  # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> SHIFT32, p0 & MASK32
        hi1, lo1 = p1 >> SHIFT32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox_for_groups(seed, groups):
    """Philox4x32-10 words for the given 64-bit group counters under ``seed``.

    Counter = (g_lo, g_hi, 0, 0), key = (seed_lo, seed_hi). Returns an
    array of shape (len(groups), 4) of uint32.
    """
    g = np.asarray(groups, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64(seed >> 32)
    r = philox4x32(g & MASK32, g >> SHIFT32, 0, 0, k0, k1)
    return np.stack([x.astype(np.uint32) for x in r], axis=-1)
