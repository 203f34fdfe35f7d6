"""Power spectrum and moments of a field on the periodic grid (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.1: the tool that builds the velocity fields prints basic statistics of
the white noise and of the fields, and can output the density field and the
power spectrum measured from it. The estimator (the paper does not spell it
out; this is the standard one):

  F(k)  = sum_x f(x) exp(-i k.x)                 (unnormalised DFT)
  P(b)  = (V / N^6) <|F(k)|^2>_{k in shell b}    (V = L^3)
  shell b: b = floor(|m| + 1/2), the smallest b with 4 m^2 < (2b + 1)^2
           (m^2 = m_x^2 + m_y^2 + m_z^2), b = 0 .. nbins - 1;
  k(b)  = mean of |k| = 2 pi |m| / L over the shell's modes.

Modes with any |m_j| = N/2 are left out, as everywhere on this path. The
average runs over all modes of the full spectrum: on the half spectrum a
mode with 0 < m_z < N/2 stands for itself and its conjugate partner
(weight 2), one with m_z = 0 for itself (its partner is stored too). For a
unit-variance white noise <P(b)> = V / N^3 for every shell but b = 0, and for
delta = sqrt(P/V) W-tilde, i.e. the Eq. 1 field, <P(b)> = D^2 P(k).

Moments: mean, variance (population, FP64 two-pass), minimum, maximum.
"""
import numpy as np

from . import fields


def shells(n):
    """Shell index b of every half-spectrum mode (-1 where left out) and its weight."""
    mx, my, mz = fields.integer_modes(n)
    m2 = (mx * mx + my * my + mz * mz).astype(np.int64)
    b = np.floor(np.sqrt(m2.astype(np.float64)) + 0.5).astype(np.int64)
    # exact integer shell test (the float estimate is off by at most one)
    b = np.where((2 * b + 1) ** 2 <= 4 * m2, b + 1, b)
    b = np.where((b > 0) & (4 * m2 < (2 * b - 1) ** 2), b - 1, b)
    ny = n // 2
    out = (np.abs(mx) == ny) | (np.abs(my) == ny) | (mz == ny)
    b = np.where(out, -1, b)
    w = np.where(mz == 0, 1, 2) * np.ones_like(b)
    return b, w, m2


def power_spectrum(field, box, nbins):
    """(k, P, count) per shell b < nbins; count = modes of the full spectrum."""
    f = np.asarray(field, dtype=np.float64)
    n = f.shape[0]
    fk = np.fft.rfftn(f)
    b, w, m2 = shells(n)
    sel = (b >= 0) & (b < nbins)
    bb, ww = b[sel], w[sel]
    p2 = (np.abs(fk) ** 2)[sel]
    kk = (2 * np.pi / box) * np.sqrt(m2[sel].astype(np.float64))
    cnt = np.bincount(bb, weights=ww, minlength=nbins)[:nbins]
    sp = np.bincount(bb, weights=ww * p2, minlength=nbins)[:nbins]
    sk = np.bincount(bb, weights=ww * kk, minlength=nbins)[:nbins]
    vol = box ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        p = np.where(cnt > 0, vol / float(n) ** 6 * sp / cnt, 0.0)
        k = np.where(cnt > 0, sk / cnt, 0.0)
    return k, p, cnt.astype(np.int64)


def moments(field):
    """(mean, variance, min, max) in FP64."""
    f = np.asarray(field, dtype=np.float64).ravel()
    m = f.mean()
    return m, float(np.mean((f - m) ** 2)), float(f.min()), float(f.max())
