"""Pins of the oracle's Eqs. 1-3 path against brute-force sums and closed forms.

* the forward transform and its normalisation against an explicit O(N^6)
  DFT (8^3, 12^3);
* psi_j (Eq. 2) against an explicit full-grid inverse sum built from the
  full (not half) spectrum, which fixes the Hermitian and Nyquist handling;
* a planted Fourier mode, whose delta and psi are known in closed form;
* div psi = -delta and curl psi = 0 for random noise;
* Parseval on the half spectrum;
* the measured power spectrum of many realizations against the input P(k).
"""
import math

import numpy as np
import pytest

from oracle import fields
from oracle.noise import white_noise
from tests.oracle_cases import BBKS, cosmology_from

COSMO = cosmology_from(BBKS)


def _dft_matrix_3d(n, sign):
    i = np.arange(n)
    ix, iy, iz = np.meshgrid(i, i, i, indexing="ij")
    x = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1)  # (N^3, 3)
    phase = (x @ x.T) % n  # k.x for k and x on the same integer grid
    return np.exp(sign * 2j * np.pi * phase / n)


@pytest.mark.parametrize("n", [8, 12])
def test_forward_transform_brute_force(n):
    w = np.random.default_rng(n).standard_normal((n, n, n))
    full = (_dft_matrix_3d(n, -1) @ w.ravel()).reshape(n, n, n) / n ** 1.5
    got = fields.spectrum(w)
    want = full[:, :, : n // 2 + 1]
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("n", [8, 12])
def test_psi_brute_force_full_grid(n):
    box, z = 50.0, 30.0
    w = np.random.default_rng(100 + n).standard_normal((n, n, n))
    out = fields.zeldovich(n, box, COSMO, z, noise=w, want_delta=True)
    d = out["D"]
    # full spectrum by explicit DFT, full-grid filter built from the definition
    wk = (_dft_matrix_3d(n, -1) @ w.ravel()) / n ** 1.5
    i = np.arange(n)
    m = np.where(i < n // 2, i, i - n)
    mx, my, mz = np.meshgrid(m, m, m, indexing="ij")
    mvec = np.stack([mx.ravel(), my.ravel(), mz.ravel()], 1).astype(float)
    m2 = (mvec ** 2).sum(1)
    drop = (m2 == 0) | np.any(np.abs(mvec) == n // 2, axis=1)
    k = 2 * math.pi / box * np.sqrt(m2)
    p = np.zeros_like(k)
    p[~drop] = COSMO.power(k[~drop])
    s = np.where(drop, 0.0, d * np.sqrt(p / box ** 3))
    inv = _dft_matrix_3d(n, +1)
    delta = inv @ (s * wk)
    assert np.max(np.abs(delta.imag)) < 1e-13 * np.max(np.abs(delta.real))
    np.testing.assert_allclose(out["delta"].ravel(), delta.real, rtol=0, atol=1e-12 * np.abs(delta).max())
    for j in range(3):
        kj = 2 * math.pi / box * mvec[:, j]
        with np.errstate(invalid="ignore", divide="ignore"):
            h = np.where(drop, 0.0, kj / (2 * math.pi / box) ** 2 / np.where(m2 > 0, m2, 1.0))
        psi = inv @ (1j * h * s * wk)
        assert np.max(np.abs(psi.imag)) < 1e-13 * np.max(np.abs(psi.real))
        np.testing.assert_allclose(out["psi"][j].ravel(), psi.real, rtol=0,
                                   atol=1e-12 * np.abs(psi).max())


@pytest.mark.parametrize("m0", [(1, -2, 3), (0, 0, 5), (7, 1, -1), (-3, 6, 0)])
def test_planted_mode_closed_form(m0):
    n, box, z = 16, 100.0, 50.0
    i = np.arange(n)
    ix, iy, iz = np.meshgrid(i, i, i, indexing="ij")
    phase = 2 * math.pi * (m0[0] * ix + m0[1] * iy + m0[2] * iz) / n
    out = fields.zeldovich(n, box, COSMO, z, noise=np.cos(phase), want_delta=True)
    k0 = 2 * math.pi / box * np.array(m0, dtype=float)
    kk = math.sqrt((k0 ** 2).sum())
    s = out["D"] * math.sqrt(COSMO.power(kk) * n ** 3 / box ** 3)
    np.testing.assert_allclose(out["delta"], s * np.cos(phase), atol=1e-12 * s)
    for j in range(3):
        want = -s * k0[j] / kk ** 2 * np.sin(phase)
        np.testing.assert_allclose(out["psi"][j], want, atol=1e-12 * s / kk)
    # particles move towards the density crests: psi . grad(delta) >= 0 where it is not zero
    gx = -s * k0[0] * np.sin(phase)
    assert np.all(out["psi"][0] * gx >= -1e-12 * s * s)


def _spectral_derivative(f, box, j):
    n = f.shape[0]
    mx, my, mz = fields.integer_modes(n)
    kj = 2 * math.pi / box * [mx, my, mz][j]
    fk = np.fft.rfftn(f)
    fk = np.where(np.abs([mx, my, mz][j]) == n // 2, 0, fk)
    return np.fft.irfftn(1j * kj * fk, s=f.shape, axes=(0, 1, 2))


def test_div_curl_identities():
    n, box = 32, 64.0
    out = fields.zeldovich(n, box, COSMO, 20.0, seed=3, want_delta=True)
    psi = out["psi"]
    div = sum(_spectral_derivative(psi[j], box, j) for j in range(3))
    scale = np.abs(out["delta"]).max()
    assert np.max(np.abs(div + out["delta"])) < 1e-12 * scale
    for a, b in ((0, 1), (1, 2), (0, 2)):
        curl = _spectral_derivative(psi[b], box, a) - _spectral_derivative(psi[a], box, b)
        assert np.max(np.abs(curl)) < 1e-12 * scale


def test_parseval_half_spectrum():
    n = 24
    w = white_noise(2, n)
    wk = fields.spectrum(w)
    weight = np.full(wk.shape, 2.0)
    weight[:, :, 0] = 1.0
    weight[:, :, n // 2] = 1.0
    assert abs((weight * np.abs(wk) ** 2).sum() - (w ** 2).sum()) < 1e-10 * (w ** 2).sum()


def test_linear_in_noise():
    n, box = 16, 40.0
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal((2, n, n, n))
    fa = fields.zeldovich(n, box, COSMO, 10.0, noise=a)["psi"][1]
    fb = fields.zeldovich(n, box, COSMO, 10.0, noise=b)["psi"][1]
    fab = fields.zeldovich(n, box, COSMO, 10.0, noise=2 * a - 3 * b)["psi"][1]
    np.testing.assert_allclose(fab, 2 * fa - 3 * fb, atol=1e-13 * np.abs(fab).max())


def test_measured_power_matches_input():
    """Mean of V |delta~|^2 / (D^2 P(k)) over modes and realizations is 1 per shell."""
    n, box, reals = 32, 200.0, 40
    mx, my, mz = fields.integer_modes(n)
    m2 = (mx * mx + my * my + mz * mz)
    keep = fields.keep_mask(n) & (mz > 0)  # kz > 0: every mode independent
    k = 2 * math.pi / box * np.sqrt(m2.astype(float))
    pk = np.where(keep, COSMO.power(np.where(keep, k, 1.0)), 1.0)
    shells = np.floor(np.sqrt(m2)).astype(int)
    sums = np.zeros(n)
    counts = np.zeros(n)
    for r in range(reals):
        out = fields.zeldovich(n, box, COSMO, 0.0, seed=1000 + r, want_delta=True, components=())
        dk = np.fft.rfftn(out["delta"]) / n ** 3
        ratio = box ** 3 * np.abs(dk) ** 2 / (out["D"] ** 2 * pk)
        np.add.at(sums, shells[keep], ratio[keep])
        np.add.at(counts, shells[keep], 1)
    use = counts > 0
    mean = sums[use] / counts[use]
    assert np.all(np.abs(mean - 1.0) < 5.0 / np.sqrt(counts[use]))


def test_velocity_and_positions():
    n, box = 16, 30.0
    out = fields.zeldovich(n, box, COSMO, 49.0, seed=1)
    q = fields.lattice(n, box)
    for j in range(3):
        ratio = out["vel"][j][out["psi"][j] != 0] / out["psi"][j][out["psi"][j] != 0]
        assert np.allclose(ratio, out["vfac"], rtol=1e-15)
        pos = out["pos"][j]
        assert pos.min() >= 0.0 and pos.max() < box
        sh = [1, 1, 1]
        sh[j] = n
        disp = pos - q.reshape(sh)
        disp = disp - box * np.round(disp / box)
        np.testing.assert_allclose(disp, out["psi"][j], atol=1e-12 * box)
    assert abs(q[0] - 0.5 * box / n) < 1e-15
