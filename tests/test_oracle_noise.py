"""Pins of the oracle's white noise: Box-Muller special values and statistics.

The paper asks for independent Gaussian numbers of zero mean and unit
variance (Sec. 2, step 1). The closed-form cases below fix the uniform
mapping, the lane-to-word assignment and the cos/sin split; the statistical
tests fix the distribution.
"""
import math

import numpy as np
from scipy import stats

from oracle import noise
from oracle.philox import philox_for_groups


def _words(ra, rb, rc, rd):
    return np.array([[ra, rb, rc, rd]], dtype=np.uint32)


def test_unit_uniform_gives_zero():
    # r_a = 2^32 - 1 -> u_a = 1 -> rho = 0
    w = noise.gaussian_from_words(_words(0xFFFFFFFF, 123, 0xFFFFFFFF, 5), [0])
    assert w[0] == 0.0


def test_half_uniform_and_quarter_turn():
    # r_a = 2^31 - 1 -> u_a = 1/2 -> rho = sqrt(2 ln 2); r_b = 2^30 -> angle pi/2
    rho = math.sqrt(2.0 * math.log(2.0))
    words = _words(2**31 - 1, 2**30, 2**31 - 1, 2**29)
    even0, odd0 = noise.gaussian_from_words(np.repeat(words, 2, 0), [0, 1])
    assert abs(even0) < 1e-15 and abs(odd0 - rho) < 1e-15
    # pair 1 (lanes 2, 3) uses words 2, 3: angle pi/4 -> cos = sin = 1/sqrt(2)
    even1, odd1 = noise.gaussian_from_words(np.repeat(words, 2, 0), [2, 3])
    assert abs(even1 - rho / math.sqrt(2.0)) < 1e-15
    assert abs(odd1 - rho / math.sqrt(2.0)) < 1e-15


def test_zero_angle():
    # r_b = 0 -> cos 0 = 1, sin 0 = 0; r_a = 0 -> u_a = 2^-32
    rho = math.sqrt(64.0 * math.log(2.0))
    w = noise.gaussian_from_words(np.repeat(_words(0, 0, 0, 0), 2, 0), [0, 1])
    assert abs(w[0] - rho) < 1e-14 and w[1] == 0.0


def test_cell_uses_its_group_and_lane():
    seed = 11
    idx = np.array([0, 1, 2, 3, 4, 5, 4 * 1000 + 2, 2**33 + 3], dtype=np.int64)
    got = noise.noise_at(seed, idx)
    for i, v in zip(idx, got):
        words = philox_for_groups(seed, [int(i) >> 2])
        assert v == noise.gaussian_from_words(words, [int(i) & 3])[0]


def test_grid_is_cell_index_function():
    n = 6
    w = noise.white_noise(5, n)
    ix, iy, iz = 2, 3, 4
    assert w[ix, iy, iz] == noise.noise_at(5, [(ix * n + iy) * n + iz])[0]


def test_gaussian_moments():
    x = noise.noise_at(7, np.arange(1 << 22, dtype=np.int64))
    n = x.size
    assert abs(x.mean()) < 5 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.skew(x)) < 5 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(x)) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(x[: 1 << 20], "norm").pvalue > 1e-4


def test_neighbours_uncorrelated():
    x = noise.noise_at(9, np.arange(1 << 21, dtype=np.int64))
    n = x.size - 1
    for lag in (1, 2, 3, 4):
        c = np.mean(x[:-lag] * x[lag:])
        assert abs(c) < 5 / math.sqrt(n)
    # cos/sin partners of one Box-Muller pair are independent: E[W0^2 W1^2] = 1
    pairs = x.reshape(-1, 2)
    assert abs(np.mean(pairs[:, 0] ** 2 * pairs[:, 1] ** 2) - 1.0) < 5 * math.sqrt(8.0 / pairs.shape[0])


def test_seeds_differ():
    a = noise.noise_at(1, np.arange(4096))
    b = noise.noise_at(2, np.arange(4096))
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / 64
