"""Gaussian white noise keyed by (seed, global cell index) (oracle).

Paper: Sec. 2, step 1 -- the white noise (WN) field is a grid of independent
Gaussian numbers with zero mean and unit variance; Sec. 2.1 draws them from
SPRNG. Reading taken here (the paper fixes no generator): Philox4x32-10 plus
the two-output Box-Muller transform (G. E. P. Box, M. E. Muller, Ann. Math.
Statist. 29, 610 (1958)).

Cell index (C order, z fastest):  idx = (i_x * N + i_y) * N + i_z.
Four consecutive cells share one Philox call:
    g    = idx >> 2      group counter, Philox counter (g_lo, g_hi, 0, 0)
    lane = idx & 3       key = (seed_lo, seed_hi)
Pair p = lane >> 1 uses the words (r_{2p}, r_{2p+1}):
    u_a = (r_{2p} + 1) * 2^-32   in (0, 1]
    u_b = r_{2p+1} * 2^-32       in [0, 1)
    rho = sqrt(-2 ln u_a)
    W   = rho * cos(2 pi u_b)   for even lanes,   rho * sin(2 pi u_b) for odd.
The value depends only on (seed, idx): never on the launch shape or on
batching. The same seed on grids of different N reuses counters.
"""
import numpy as np

from .philox import philox_for_groups

TWO_M32 = 2.0 ** -32


def gaussian_from_words(words, lanes):
    """Box-Muller value for each cell from its group's four Philox words.

    ``words``: (n, 4) uint32 Philox outputs of each cell's group; ``lanes``:
    (n,) cell lane in 0..3. FP64 throughout.
    """
    words = np.asarray(words, dtype=np.uint64)
    lanes = np.asarray(lanes, dtype=np.int64)
    p = lanes >> 1
    ra = np.take_along_axis(words, (2 * p)[:, None], axis=1)[:, 0]
    rb = np.take_along_axis(words, (2 * p + 1)[:, None], axis=1)[:, 0]
    ua = (ra.astype(np.float64) + 1.0) * TWO_M32
    ub = rb.astype(np.float64) * TWO_M32
    rho = np.sqrt(-2.0 * np.log(ua))
    ang = 2.0 * np.pi * ub
    return np.where((lanes & 1) == 0, rho * np.cos(ang), rho * np.sin(ang))


def noise_at(seed, idx):
    """W at arbitrary global cell indices (1-D int array), FP64."""
    idx = np.asarray(idx, dtype=np.int64)
    words = philox_for_groups(seed, (idx >> 2).astype(np.uint64))
    return gaussian_from_words(words, idx & 3)


def noise_bits(seed, groups):
    """Raw Philox words (n, 4) uint32 for the given group counters."""
    return philox_for_groups(seed, groups)


def white_noise(seed, n, chunk=1 << 22):
    """The full N^3 white-noise grid W[i_x, i_y, i_z] in FP64."""
    total = n ** 3
    out = np.empty(total, dtype=np.float64)
    for s in range(0, total, chunk):
        e = min(total, s + chunk)
        out[s:e] = noise_at(seed, np.arange(s, e, dtype=np.int64))
    return out.reshape(n, n, n)
