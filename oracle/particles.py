"""Particle-set options of the Eq. 3 epilogue (Sec. 2.2) and the degraded
velocity field (Sec. 2.4) (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2 (particle generation):
* periodic shift: every position moves by a fixed vector s, modulo L (to put
  a zoom region at the box centre);
* gas particles: each dark-matter particle gets a gas partner offset by half
  a cell along each axis, and both move so that the pair's centre of mass
  stays at the original particle. With the gas mass fraction f (Omega_b /
  Omega_m) the partners sit at x - f d and x + (1 - f) d, d = (Delta/2)(1,1,1);
  both carry the particle's velocity;
* coordinate-based IDs: an ID from which the Lagrangian position follows,
  also across the levels of a zoom.
Sec. 2.4 (degrading): nearest-grid-point sampling of a fine field, then a
translation in Fourier space that puts the samples at the coarse cell
centres.

Readings taken where the text is silent:
* Positions as in ``fields.zeldovich``: x = (q + s + psi) mod L, the gas and
  dark-matter offsets added to q as well.
* IDs: with n_f points per axis on the finest grid of the simulation (a
  multiple r of this grid's N), a particle at Lagrangian cell (i, j, k) gets
  offset + (I n_f + J) n_f + K, (I, J, K) = r (i, j, k) + floor(r / 2), the
  finest cell containing its Lagrangian position (the cell centre). Decoding
  gives that finest cell: the Lagrangian position is its centre for odd r
  and its lower corner for even r.
* Degrading by an integer factor r: coarse cell i takes the fine value at
  index r i (nearest grid point), whose centre lies t = (r - 1) / (2 r)
  coarse cells before the coarse cell centre; the coarse field is moved by
  that fraction of a cell in Fourier space (exact for band-limited fields).
  The text's "half a low-resolution cell" is the same move for grid values
  taken at the cell corners. Modes with any |m_j| = N/2 are dropped, as
  everywhere on this path (a shifted Nyquist mode is not real).
"""
import numpy as np

from . import fields


def positions(psi, box, shift=(0.0, 0.0, 0.0), extra=0.0, q_offset=0.5):
    """Eq. 3 positions per axis with a periodic shift and an extra offset
    (the same on every axis): (q + shift_j + extra + psi_j) mod L."""
    n = psi[0].shape[0]
    out = []
    for j in range(3):
        sh = [1, 1, 1]
        sh[j] = n
        q = fields.lattice(n, box, q_offset).reshape(sh)
        out.append(fields.wrap(q + shift[j] + extra + psi[j], box))
    return out


def gas_pairs(psi, box, gas_fraction, shift=(0.0, 0.0, 0.0), q_offset=0.5):
    """(dark-matter positions, gas positions) of the pairs."""
    n = psi[0].shape[0]
    d = 0.5 * box / n
    dm = positions(psi, box, shift, -gas_fraction * d, q_offset)
    gas = positions(psi, box, shift, (1.0 - gas_fraction) * d, q_offset)
    return dm, gas


def particle_ids(n, n_finest, offset=0):
    """Coordinate-based IDs of the n^3 particles (int64)."""
    if n_finest % n:
        raise ValueError("the finest grid must be a multiple of this grid")
    r = n_finest // n
    c = r * np.arange(n, dtype=np.int64) + r // 2
    return offset + (c[:, None, None] * n_finest + c[None, :, None]) * n_finest + c[None, None, :]


def id_to_fine_cell(ids, n_finest, offset=0):
    """The finest-grid cell (I, J, K) an ID encodes."""
    v = np.asarray(ids, dtype=np.int64) - offset
    return v // (n_finest * n_finest), (v // n_finest) % n_finest, v % n_finest


def degrade(field, r):
    """Nearest-grid-point sample of every r-th fine value, moved in Fourier
    space by t = (r - 1) / (2 r) coarse cells along each axis."""
    f = np.asarray(field, dtype=np.float64)
    nc = f.shape[0] // r
    g = f[::r, ::r, ::r]
    t = (r - 1) / (2.0 * r)
    gk = np.fft.rfftn(g)
    mx, my, mz = fields.integer_modes(nc)
    keep = (np.abs(mx) != nc // 2) & (np.abs(my) != nc // 2) & (mz != nc // 2)
    phase = np.exp(2j * np.pi * t * (mx + my + mz) / nc)
    return np.fft.irfftn(np.where(keep, gk * phase, 0.0), s=g.shape, axes=(0, 1, 2))
