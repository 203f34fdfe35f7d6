"""Pins of the oracle's particle-set options and the degraded field.

* gas pairs: the mass-weighted centre of each pair is the original particle
  position and the partners are half a cell apart on every axis;
* periodic shift: positions move by the shift vector modulo L;
* IDs: unique, and decoding gives the finest cell holding the Lagrangian
  position (plain linear index when the grid is the finest);
* degrading: for a field band-limited below the coarse Nyquist frequency,
  the degraded samples equal the field at the coarse cell centres.
"""
import numpy as np
import pytest

from oracle import fields, particles
from oracle import noise as onoise


def _mi(d, box):
    return d - box * np.round(d / box)


def test_gas_pairs_keep_centre_of_mass():
    n, box, f = 12, 30.0, 0.157
    rng = np.random.default_rng(0)
    psi = [rng.standard_normal((n, n, n)) * 2.0 for _ in range(3)]
    base = particles.positions(psi, box)
    dm, gas = particles.gas_pairs(psi, box, f)
    for j in range(3):
        com = base[j] + (1 - f) * _mi(dm[j] - base[j], box) + f * _mi(gas[j] - base[j], box)
        assert np.abs(_mi(com - base[j], box)).max() < 1e-12
        assert np.abs(_mi(gas[j] - dm[j], box) - 0.5 * box / n).max() < 1e-12
        assert dm[j].min() >= 0 and dm[j].max() < box and gas[j].max() < box


def test_periodic_shift():
    n, box = 8, 10.0
    rng = np.random.default_rng(1)
    psi = [rng.standard_normal((n, n, n)) for _ in range(3)]
    s = (3.5, -12.25, 9.75)
    a, b = particles.positions(psi, box), particles.positions(psi, box, shift=s)
    for j in range(3):
        assert np.abs(_mi(b[j] - a[j] - s[j], box)).max() < 1e-12
        assert b[j].min() >= 0 and b[j].max() < box


@pytest.mark.parametrize("n,nf", [(8, 8), (8, 16), (6, 18), (4, 32)])
def test_ids_decode_to_lagrangian_cell(n, nf):
    ids = particles.particle_ids(n, nf, offset=1000)
    assert np.unique(ids).size == n ** 3
    if n == nf:
        assert np.array_equal(ids - 1000, np.arange(n ** 3).reshape(n, n, n))
    box = 1.0
    fi, fj, fk = particles.id_to_fine_cell(ids, nf, offset=1000)
    q = fields.lattice(n, box)  # cell centres
    want = np.floor(q * nf / box + 1e-9).astype(np.int64)
    assert np.array_equal(fi[:, 0, 0], want) and np.array_equal(fj[0, :, 0], want)
    assert np.array_equal(fk[0, 0, :], want)


@pytest.mark.parametrize("r", [2, 3])
def test_degrade_band_limited_field_exactly(r):
    nc, box = 12, 50.0
    nf = r * nc
    modes = [((1, 2, -3), 0.7, 0.3), ((4, 0, 1), -0.4, 1.1), ((0, -5, 2), 0.25, -0.6)]
    def field(nn):
        x = (np.arange(nn) + 0.5) * box / nn
        out = np.zeros((nn, nn, nn))
        for m, a, ph in modes:
            k = 2 * np.pi * np.array(m) / box
            out += a * np.cos(k[0] * x[:, None, None] + k[1] * x[None, :, None]
                              + k[2] * x[None, None, :] + ph)
        return out
    got = particles.degrade(field(nf), r)
    assert np.abs(got - field(nc)).max() < 1e-12


def test_degrade_by_one_drops_only_nyquist_modes():
    # r = 1 is the identity up to the dropped Nyquist modes
    f = onoise.white_noise(3, 8)
    g = particles.degrade(f, 1)
    fk = np.fft.rfftn(f)
    mx, my, mz = fields.integer_modes(8)
    keep = (np.abs(mx) != 4) & (np.abs(my) != 4) & (mz != 4)
    want = np.fft.irfftn(np.where(keep, fk, 0), s=f.shape, axes=(0, 1, 2))
    assert np.abs(g - want).max() < 1e-13
