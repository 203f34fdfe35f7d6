"""Pins of the oracle's power spectrum and moments.

* shell mode counts against a brute-force enumeration of the full spectrum;
* a planted cosine: all power in its shell, P = V A^2 / (2 count) there;
* white noise: <P> = V / N^3 (mean over shells within its sampling error);
* the Eq. 1 field: P(b) against the shell average of D^2 P(k) of the input
  spectrum, within the per-shell sampling error;
* moments of a two-valued field in closed form.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import fields, noise, stats
from tests.oracle_cases import BBKS, cosmology_from


@pytest.mark.parametrize("n", [6, 8, 12])
def test_shell_counts_brute_force(n):
    nb = n // 2
    _, _, cnt = stats.power_spectrum(np.zeros((n, n, n)), 1.0, nb)
    want = np.zeros(nb, dtype=np.int64)
    rng = range(-(n // 2) + 1, n // 2)  # |m_j| = N/2 left out
    for m in itertools.product(rng, repeat=3):
        m2 = sum(v * v for v in m)
        b = 0
        while not 4 * m2 < (2 * b + 1) ** 2:  # b = floor(|m| + 1/2)
            b += 1
        if b < nb:
            want[b] += 1
    assert np.array_equal(cnt, want)


def test_planted_cosine():
    n, box, amp = 16, 40.0, 0.7
    m0 = (2, -1, 3)
    x = np.arange(n) * box / n
    k = 2 * np.pi * np.array(m0) / box
    f = amp * np.cos(k[0] * x[:, None, None] + k[1] * x[None, :, None] + k[2] * x[None, None, :] + 0.3)
    kk, p, cnt = stats.power_spectrum(f, box, n // 2)
    b0 = int(math.floor(math.sqrt(sum(v * v for v in m0)) + 0.5))
    want = box ** 3 * amp * amp / (2 * cnt[b0])
    assert abs(p[b0] - want) < 1e-12 * want
    assert np.abs(np.delete(p, b0)).max() < 1e-20 * want


def test_white_noise_is_flat():
    n, box = 48, 100.0
    kk, p, cnt = stats.power_spectrum(noise.white_noise(5, n), box, n // 2)
    ratio = p[1:] * n ** 3 / box ** 3
    modes = cnt[1:].sum()
    # mode-weighted mean of |W~|^2 (exponential per complex mode, pairs identical)
    mean = np.sum(ratio * cnt[1:]) / modes
    assert abs(mean - 1) < 5 * math.sqrt(2.0 / modes)


def test_eq1_field_follows_input_spectrum():
    n, box, z = 64, 200.0, 10.0
    c = cosmology_from(BBKS)
    out = fields.zeldovich(n, box, c, z, seed=8, want_delta=True, components=())
    kk, p, cnt = stats.power_spectrum(out["delta"], box, n // 2)
    # the input spectrum averaged over the same modes
    b, w, m2 = stats.shells(n)
    sel = (b >= 1) & (b < n // 2)
    kmode = 2 * np.pi / box * np.sqrt(m2[sel].astype(np.float64))
    pin = out["D"] ** 2 * c.power(kmode)
    want = np.bincount(b[sel], weights=w[sel] * pin, minlength=n // 2)[: n // 2]
    want = want / np.maximum(cnt, 1)
    for s in range(4, n // 2):
        assert abs(p[s] / want[s] - 1) < 5 * math.sqrt(2.0 / cnt[s]), s


def test_moments_closed_form():
    f = np.where((np.indices((4, 4, 4)).sum(axis=0) % 2) == 0, 1.0, -1.0)
    assert stats.moments(f) == (0.0, 1.0, -1.0, 1.0)
