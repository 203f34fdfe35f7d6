"""Large scales of a low-resolution field plus small scales of a
high-resolution one (Sec. 2.4, Eqs. 4-5) (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.4 combines the velocity fields of a low-resolution white noise and of
its refined high-resolution version: the small scales come from the
high-resolution field through a spherical top hat in k (Eq. 4),
v_small(k) = v_high(k) (1 - f(|k| r_s)), f(x) = 1 for x < 1 else 0; the
large scales come from the low-resolution field (Eq. 5),
v_large(k) = v_low(k) f(|k| r_s). The large-scale part lives on the coarse
grid: it is divided by the Fourier transform of the cloud-in-cell kernel,
interpolated to the fine grid with cloud-in-cell weights, and added.

Readings taken where the section is silent:
* k is the angular wavenumber 2 pi m / L, so the top hat keeps the modes
  with m^2 < (L / (2 pi r_s))^2 on the low side (and m^2 >= that on the high
  side). The paper's cutoff is r_s = 2 L / N_low.
* Grid values sit at cell centres (Sec. 2.2): coarse cell i at
  (i + 1/2) L / N_low, fine cell i' at (i' + 1/2) L / N_high. Cloud-in-cell
  interpolation is the trilinear interpolation between the eight coarse cell
  centres around a fine cell centre (periodic).
* Its transform: linear interpolation per axis is the convolution with the
  triangle of half-width one coarse cell, whose transform is
  sinc^2(k_j Delta / 2) = [sin(pi m_j / N_low) / (pi m_j / N_low)]^2; the
  deconvolution divides by the product over the three axes.
* Modes with any |m_j| = N/2 are dropped, as everywhere on this path (they
  matter only for cutoffs below about a third of a cell).
* The Zel'dovich epilogue (Eq. 3) is applied to the merged displacement,
  so positions and velocities follow from it as in ``fields.zeldovich``.
"""
import numpy as np

from . import fields


def low_modes(n, box, r_s):
    """f(|k| r_s) on the half spectrum: True where |k| r_s < 1 (Eq. 5)."""
    mx, my, mz = fields.integer_modes(n)
    m2 = (mx * mx + my * my + mz * mz).astype(np.float64)
    return (2.0 * np.pi / box) ** 2 * m2 * r_s * r_s < 1.0


def cic_window(n):
    """prod_j [sin(pi m_j / N) / (pi m_j / N)]^2 on the half spectrum."""
    mx, my, mz = fields.integer_modes(n)
    s = lambda m: np.sinc(m.astype(np.float64) / n) ** 2  # np.sinc(x) = sin(pi x) / (pi x)
    return s(mx) * s(my) * s(mz)


def large_scales(field, box, r_s):
    """Eq. 5 with the deconvolution: F^-1[f(|k| r_s) F[field] / W_CIC]."""
    n = field.shape[0]
    fk = np.fft.rfftn(np.asarray(field, dtype=np.float64))
    mx, my, mz = fields.integer_modes(n)
    no_nyquist = (np.abs(mx) != n // 2) & (np.abs(my) != n // 2) & (mz != n // 2)
    fk = np.where(low_modes(n, box, r_s) & no_nyquist, fk / cic_window(n), 0.0)
    return np.fft.irfftn(fk, s=field.shape, axes=(0, 1, 2))


def cic_coordinates(n_low, n_high):
    """Per fine cell along one axis: first coarse cell (periodic) and weight
    of the second, for the fine cell centre in coarse cell-centre units."""
    u = (np.arange(n_high, dtype=np.float64) + 0.5) * n_low / n_high - 0.5
    i0 = np.floor(u).astype(np.int64)
    return np.mod(i0, n_low), u - i0


def cic_interpolate(field_low, n_high):
    """Trilinear (cloud-in-cell) interpolation of a periodic coarse grid to
    the cell centres of a fine grid of n_high points per axis."""
    c = np.asarray(field_low, dtype=np.float64)
    n_low = c.shape[0]
    i0, t = cic_coordinates(n_low, n_high)
    i1 = np.mod(i0 + 1, n_low)
    out = np.zeros((n_high, n_high, n_high))
    for cx, wx in ((i0, 1.0 - t), (i1, t)):
        for cy, wy in ((i0, 1.0 - t), (i1, t)):
            for cz, wz in ((i0, 1.0 - t), (i1, t)):
                out += (c[np.ix_(cx, cy, cz)] * wx[:, None, None] * wy[None, :, None]
                        * wz[None, None, :])
    return out


def merged_zeldovich(n, box, cosmo, z_init, large, r_s, seed=None, noise=None, q_offset=0.5):
    """Eq. 4 on the fine-grid displacement of ``noise`` (or ``seed``), plus the
    interpolated coarse large scales ``large`` (three coarse grids, Eq. 5 with
    the deconvolution already applied, e.g. by ``large_scales``), then Eq. 3.
    Returns psi, pos, vel dicts as ``fields.zeldovich``."""
    a = 1.0 / (1.0 + z_init)
    growth, vfac = cosmo.growth(a), cosmo.velocity_factor(a)
    w = fields.white_noise(seed, n) if noise is None else np.asarray(noise, dtype=np.float64)
    d_hat = fields.delta_hat(fields.spectrum(w), box, cosmo, growth)
    high = ~low_modes(n, box, r_s)
    out = {"psi": {}, "pos": {}, "vel": {}, "vfac": vfac}
    for j in range(3):
        small = fields.to_real(np.where(high, fields.psi_hat(d_hat, box, j), 0.0), n)
        psi = small + cic_interpolate(large[j], n)
        sh = [1, 1, 1]
        sh[j] = n
        q = fields.lattice(n, box, q_offset).reshape(sh)
        out["psi"][j] = psi
        out["pos"][j] = fields.wrap(q + psi, box)
        out["vel"][j] = vfac * psi
    return out
