"""Eqs. 1-3 of the paper on a periodic N^3 grid (oracle, FP64).

Sec. 2.1, Eq. 1:   delta~(k) = sqrt(P(|k|)) W~(k)
Sec. 2.1, Eq. 2:   v~_j(k)   = i delta~(k) k_j / |k|^2
Sec. 2.2, Eq. 3:   x_j = q_j - D/(a Ddot) v_j   (Zel'dovich approximation)

Readings taken where the paper is silent:

* Transform conventions. Forward transform orthonormal,
  W~(k) = N^{-3/2} sum_x W(x) exp(-i k.x); inverse unnormalised,
  f(x) = sum_k f~(k) exp(+i k.x); the filter carries sqrt(P/V), V = L^3.
  Then <delta^2> = (1/V) sum_{k != 0} P(k) D^2.
* Growth. delta~ = D(z) sqrt(P(k, z=0)/V) W~, so psi carries D(z).
* Sign. psi~_j = i k_j delta~ / k^2 gives div psi = -delta (mass
  conservation, particles move towards overdensities); positions are
  x = q + psi. Eq. 3's minus sign belongs to the opposite FFT sign
  convention with v measured in velocity units.
* Nyquist and k = 0. Every mode with any |m_j| = N/2, and k = 0, is zeroed
  (i psi~ is odd in k and cannot stay Hermitian at the Nyquist plane).
* Lattice. q_j = (i_j + 1/2) Delta, the cell centre (Sec. 2.2: velocity
  components at the centre of each grid cell); ``q_offset=0`` gives the
  corner lattice.
* Velocity. v_j = 100 a E(a) f(a) psi_j km/s (psi in Mpc/h).

The FFTs are library calls (scipy.fft); nothing is blocked, fused or
reordered beyond the equations.
"""
import os

import numpy as np
import scipy.fft as sfft

from .noise import white_noise

WORKERS = max(1, len(os.sched_getaffinity(0)))


def integer_modes(n):
    """Integer frequencies m_x, m_y (full) and m_z (half, 0..N/2) in rfftn layout."""
    m = np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)
    mz = np.arange(n // 2 + 1, dtype=np.int64)
    return m[:, None, None], m[None, :, None], mz[None, None, :]


def spectrum(w):
    """W~ = N^{-3/2} rfftn(W): orthonormal forward transform (half spectrum)."""
    n = w.shape[0]
    return sfft.rfftn(w, workers=WORKERS) / n ** 1.5


def to_real(fk, n):
    """f(x) = sum_k f~(k) exp(+i k.x) from a half spectrum (unnormalised)."""
    return sfft.irfftn(fk, s=(n, n, n), norm="forward", workers=WORKERS)


def keep_mask(n):
    """True for modes that survive: k != 0 and no |m_j| = N/2."""
    mx, my, mz = integer_modes(n)
    ny = n // 2
    keep = (np.abs(mx) != ny) & (np.abs(my) != ny) & (mz != ny)
    keep = keep & ~((mx == 0) & (my == 0) & (mz == 0))
    return keep


def k_magnitude(n, box):
    mx, my, mz = integer_modes(n)
    m2 = mx * mx + my * my + mz * mz
    return 2.0 * np.pi / box * np.sqrt(m2.astype(np.float64))


def density_filter(n, box, cosmo, growth):
    """S_delta(k) = D sqrt(P(|k|)/V) on the half spectrum, zero where dropped (Eq. 1)."""
    k = k_magnitude(n, box)
    keep = keep_mask(n)
    p = np.zeros_like(k)
    p[keep] = cosmo.power(k[keep])
    return np.where(keep, growth * np.sqrt(p / box ** 3), 0.0)


def delta_hat(w_hat, box, cosmo, growth):
    """delta~(k) = S_delta(k) W~(k) (Eq. 1)."""
    n = w_hat.shape[0]
    return density_filter(n, box, cosmo, growth) * w_hat


def psi_hat(d_hat, box, j):
    """psi~_j(k) = i k_j delta~(k) / |k|^2 (Eq. 2), zero at k = 0 and Nyquist."""
    n = d_hat.shape[0]
    m = integer_modes(n)
    mx, my, mz = m
    m2 = (mx * mx + my * my + mz * mz).astype(np.float64)
    kj = 2.0 * np.pi / box * m[j].astype(np.float64)
    k2 = (2.0 * np.pi / box) ** 2 * m2
    with np.errstate(divide="ignore", invalid="ignore"):
        h = np.where(m2 > 0, kj / k2, 0.0)
    return np.where(keep_mask(n), 1j * h * d_hat, 0.0)


def lattice(n, box, q_offset=0.5):
    """Lagrangian coordinate q along one axis: (i + q_offset) * Delta."""
    return (np.arange(n, dtype=np.float64) + q_offset) * (box / n)


def wrap(x, box):
    """Periodic wrap into [0, L)."""
    y = np.mod(x, box)
    return np.where(y >= box, y - box, y)


def zeldovich(n, box, cosmo, z_init, seed=None, noise=None, q_offset=0.5,
              growth_override=None, want_delta=False, components=(0, 1, 2)):
    """The whole path: noise -> Eq. 1 -> Eq. 2 -> Eq. 3 (one component at a time).

    Returns a dict with psi[j], pos[j], vel[j] (FP64 arrays of shape (N,N,N))
    and the scalars D, f, vfac, a. ``noise`` (FP64 N^3) overrides the seed.
    """
    a = 1.0 / (1.0 + z_init)
    if growth_override is not None:
        growth, frate = growth_override
        vfac = 100.0 * a * float(cosmo.E(a)) * frate
    else:
        growth, frate = cosmo.growth(a), cosmo.growth_rate(a)
        vfac = cosmo.velocity_factor(a)
    w = white_noise(seed, n) if noise is None else np.asarray(noise, dtype=np.float64)
    d_hat = delta_hat(spectrum(w), box, cosmo, growth)
    del w
    out = {"D": growth, "f": frate, "vfac": vfac, "a": a, "psi": {}, "pos": {}, "vel": {}}
    if want_delta:
        out["delta"] = to_real(d_hat, n)
    shape = [1, 1, 1]
    for j in components:
        psi = to_real(psi_hat(d_hat, box, j), n)
        sh = list(shape)
        sh[j] = n
        q = lattice(n, box, q_offset).reshape(sh)
        out["psi"][j] = psi
        out["pos"][j] = wrap(q + psi, box)
        out["vel"][j] = vfac * psi
    return out
