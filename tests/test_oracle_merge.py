"""Pins of the oracle's large/small-scale merge (Sec. 2.4, Eqs. 4-5).

* the cloud-in-cell window against the transform of the triangle kernel by
  numerical quadrature;
* the interpolation against brute-force tent weights at fine cell centres,
  and a constant field left unchanged;
* Eq. 5 with deconvolution: modes outside the top hat vanish, modes inside
  are divided by the window; a single passband mode, deconvolved and
  interpolated, matches the continuous mode within the linear-interpolation
  error bound (k Delta)^2 / 8 plus the window's (k Delta)^2 / 12 per axis;
* Eq. 4: the small scales plus the spectral low band give back the full
  displacement of ``fields.zeldovich``;
* the method's purpose: a mode planted in the coarse noise and in its
  consistent fine counterpart is carried through the merge to the fine
  grid (low mode: within the bound above; high mode: exactly).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import fields, merge
from tests.oracle_cases import BBKS, cosmology_from

C = cosmology_from(BBKS)


def test_top_hat_threshold():
    n, box, r_s = 16, 2 * math.pi, 1.0 / math.sqrt(10.5)  # keeps m^2 < 10.5
    low = merge.low_modes(n, box, r_s)
    mx, my, mz = fields.integer_modes(n)
    m2 = mx * mx + my * my + mz * mz
    assert np.array_equal(low, m2 <= 10)


@pytest.mark.parametrize("m,n", [(1, 16), (3, 16), (5, 32), (5, 12)])
def test_cic_window_is_triangle_transform(m, n):
    # (1/D) int tri(x/D) e^{-ikx} dx with D = L/n, k = 2 pi m / L, per axis
    box = 1.0
    d = box / n
    k = 2 * math.pi * m / box
    val, _ = integrate.quad(lambda x: (1 - abs(x) / d) * math.cos(k * x), -d, d, epsabs=1e-14)
    w1 = val / d
    mx, my, mz = fields.integer_modes(n)
    win = merge.cic_window(n)
    got = win[m % n, 0, 0]
    assert abs(got - w1) < 1e-12
    assert abs(win[m % n, m % n, m] - w1 ** 3) < 1e-12


def test_interpolation_brute_force_tent_weights():
    rng = np.random.default_rng(1)
    nl, nh, box = 6, 12, 3.0
    c = rng.standard_normal((nl, nl, nl))
    got = merge.cic_interpolate(c, nh)
    dl, dh = box / nl, box / nh
    for fx, fy, fz in [(0, 0, 0), (11, 5, 2), (3, 10, 7), (6, 6, 11)]:
        x = [(f + 0.5) * dh for f in (fx, fy, fz)]
        want = 0.0
        for i in range(nl):
            for j in range(nl):
                for k in range(nl):
                    w = 1.0
                    for xa, ia in zip(x, (i, j, k)):
                        dist = abs(xa - (ia + 0.5) * dl)
                        dist = min(dist, box - dist)  # periodic
                        w *= max(0.0, 1 - dist / dl)
                    want += w * c[i, j, k]
        assert abs(got[fx, fy, fz] - want) < 1e-13


def test_interpolation_keeps_constants():
    out = merge.cic_interpolate(np.full((8, 8, 8), 2.5), 12)
    assert np.abs(out - 2.5).max() < 1e-14


def test_large_scales_spectrum():
    rng = np.random.default_rng(2)
    n, box, r_s = 16, 50.0, 50.0 / 16 * 2
    f = rng.standard_normal((n, n, n))
    got = np.fft.rfftn(merge.large_scales(f, box, r_s))
    want = np.fft.rfftn(f)
    low = merge.low_modes(n, box, r_s)
    assert np.abs(got[~low]).max() < 1e-10
    assert np.allclose(got[low], want[low] / merge.cic_window(n)[low], rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("axis,m", [(0, 1), (1, 2), (2, 1)])
def test_passband_mode_through_deconvolution_and_interpolation(axis, m):
    nl, nh, box = 32, 64, 100.0
    r_s = 2 * box / nl
    k = 2 * math.pi * m / box
    x = lambda nn: (np.arange(nn) + 0.5) * box / nn
    sh = [1, 1, 1]
    sh[axis] = -1
    coarse = np.broadcast_to(np.cos(k * x(nl)).reshape(sh), (nl, nl, nl))
    fine_exact = np.broadcast_to(np.cos(k * x(nh)).reshape(sh), (nh, nh, nh))
    got = merge.cic_interpolate(merge.large_scales(coarse, box, r_s), nh)
    kd = k * box / nl
    assert np.abs(got - fine_exact).max() < kd * kd * (1 / 8 + 1 / 12)


def test_small_scales_plus_low_band_is_full_displacement():
    n, box, z, r_s = 16, 64.0, 30.0, 2 * 64.0 / 8
    noise = fields.white_noise(4, n)
    zero = [np.zeros((8, 8, 8))] * 3
    got = merge.merged_zeldovich(n, box, C, z, zero, r_s, noise=noise)
    full = fields.zeldovich(n, box, C, z, noise=noise)
    # the spectral low band of the full displacement, added back
    low = merge.low_modes(n, box, r_s)
    for j in range(3):
        band = np.fft.irfftn(np.where(low, np.fft.rfftn(full["psi"][j]), 0.0), s=(n, n, n),
                            axes=(0, 1, 2))
        assert np.abs(got["psi"][j] + band - full["psi"][j]).max() < 1e-13 * np.abs(full["psi"][j]).max() * n


def _planted(nn, box, m0, amp):
    x = (np.arange(nn) + 0.5) * box / nn
    k = 2 * np.pi * np.asarray(m0) / box
    return amp * np.cos(k[0] * x[:, None, None] + k[1] * x[None, :, None] + k[2] * x[None, None, :])


def test_low_mode_carried_from_coarse_grid():
    nl, nh, box, z = 16, 32, 64.0, 30.0
    r_s = 2 * box / nl
    m0 = (1, 1, 0)
    # the same white-noise mode on both grids: fine cells carry (nl/nh)^{3/2}
    coarse = _planted(nl, box, m0, 1.0)
    fine = _planted(nh, box, m0, (nl / nh) ** 1.5)
    low = fields.zeldovich(nl, box, C, z, noise=coarse)
    high = fields.zeldovich(nh, box, C, z, noise=fine)
    large = [merge.large_scales(low["psi"][j], box, r_s) for j in range(3)]
    got = merge.merged_zeldovich(nh, box, C, z, large, r_s, noise=fine)
    kd = 2 * math.pi * math.sqrt(2) / box * (box / nl)
    for j in (0, 1):
        amp = np.abs(high["psi"][j]).max()
        assert np.abs(got["psi"][j] - high["psi"][j]).max() < 2 * kd * kd * (1 / 8 + 1 / 12) * amp
        assert np.abs(got["vel"][j] - high["vel"][j]).max() < 2 * kd * kd * (1 / 8 + 1 / 12) * amp * got["vfac"]


def test_high_mode_taken_from_fine_grid_exactly():
    nh, box, z = 32, 64.0, 30.0
    r_s = 2 * box / 16
    m0 = (5, 3, 2)  # |k| r_s > 1
    fine = _planted(nh, box, m0, 0.3)
    high = fields.zeldovich(nh, box, C, z, noise=fine)
    zero = [np.zeros((16, 16, 16))] * 3
    got = merge.merged_zeldovich(nh, box, C, z, zero, r_s, noise=fine)
    for j in range(3):
        assert np.abs(got["psi"][j] - high["psi"][j]).max() < 1e-12 * np.abs(high["psi"][j]).max() * nh
