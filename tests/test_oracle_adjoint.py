"""Pins of the oracle's adjoint chain (CIC density, smoothing, W -> psi transpose).

* dot products <J w, g> = <w, J^T g> for the map W -> psi (1e-12);
* CIC adjoint against central differences of the CIC density along random
  directions (FP64, h small enough that no particle crosses a node plane);
* CIC closed forms: psi = 0 or a shift by whole cells gives delta = 0, and the
  total mass is conserved; smoothing is symmetric and multiplies a planted
  mode by exp(-k^2 R^2 / 2);
* the full loss gradient against central finite differences (CIC and the
  exactly quadratic linear-density loss).
"""
import math

import numpy as np
import pytest

from oracle import adjoint
from tests.oracle_cases import BBKS, cosmology_from

C = cosmology_from(BBKS)


def test_psi_adjoint_dot_product():
    n, box, z = 12, 30.0, 20.0
    rng = np.random.default_rng(0)
    w = rng.standard_normal((n, n, n))
    g = [rng.standard_normal((n, n, n)) for _ in range(3)]
    lhs = sum(np.vdot(adjoint.psi_map(w, box, C, z, j), g[j]) for j in range(3))
    rhs = np.vdot(w, adjoint.psi_adjoint(g, box, C, z))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_cic_closed_forms():
    n, box = 8, 16.0
    zero = [np.zeros((n, n, n))] * 3
    assert np.abs(adjoint.cic_density(zero, box)).max() < 1e-15
    cell = box / n
    shift = [np.full((n, n, n), 2 * cell), np.full((n, n, n), -cell), np.zeros((n, n, n))]
    assert np.abs(adjoint.cic_density(shift, box)).max() < 1e-12
    rng = np.random.default_rng(1)
    psi = [0.7 * cell * rng.standard_normal((n, n, n)) for _ in range(3)]
    d = adjoint.cic_density(psi, box)
    assert abs(d.sum()) < 1e-10 and d.min() >= -1.0
    # half-cell shift along x: every node gets half of two particles -> delta = 0
    half = [np.full((n, n, n), 0.5 * cell), np.zeros((n, n, n)), np.zeros((n, n, n))]
    assert np.abs(adjoint.cic_density(half, box)).max() < 1e-12


def test_cic_adjoint_directional_derivative():
    n, box = 8, 16.0
    cell = box / n
    rng = np.random.default_rng(2)
    psi = [0.3 * cell * rng.standard_normal((n, n, n)) for _ in range(3)]
    g = rng.standard_normal((n, n, n))
    ga = adjoint.cic_adjoint(psi, g, box)
    for trial in range(3):
        d = [rng.standard_normal((n, n, n)) for _ in range(3)]
        h = 1e-7 * cell
        plus = adjoint.cic_density([p + h * e for p, e in zip(psi, d)], box)
        minus = adjoint.cic_density([p - h * e for p, e in zip(psi, d)], box)
        fd = np.vdot(g, (plus - minus) / (2 * h))
        an = sum(np.vdot(ga[j], d[j]) for j in range(3))
        assert abs(fd - an) < 1e-6 * abs(an)


def test_smoothing_symmetric_and_planted_mode():
    n, box, r = 16, 40.0, 3.0
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((2, n, n, n))
    assert abs(np.vdot(adjoint.smooth(a, box, r), b) - np.vdot(a, adjoint.smooth(b, box, r))) < 1e-12 * n ** 3
    i = np.arange(n)
    ix, iy, iz = np.meshgrid(i, i, i, indexing="ij")
    m = (1, 2, 3)
    f = np.cos(2 * np.pi * (m[0] * ix + m[1] * iy + m[2] * iz) / n)
    k2 = (2 * np.pi / box) ** 2 * sum(x * x for x in m)
    np.testing.assert_allclose(adjoint.smooth(f, box, r), math.exp(-0.5 * k2 * r * r) * f, atol=1e-13)


@pytest.mark.parametrize("kind,rtol", [("cic", 1e-5), ("linear", 1e-8)])
def test_loss_gradient_finite_differences(kind, rtol):
    n, box, z, radius = 16, 32.0, 50.0, 4.0
    rng = np.random.default_rng(4)
    w = rng.standard_normal((n, n, n))
    targets = rng.choice(n ** 3, size=64, replace=False)
    y = rng.standard_normal(64)
    grad = adjoint.density_loss_grad(w, box, C, z, targets, y, radius, kind)
    for c in rng.choice(n ** 3, size=6, replace=False):
        eps = 1e-3
        wp, wm = w.copy(), w.copy()
        wp.flat[c] += eps
        wm.flat[c] -= eps
        lp = adjoint.density_loss(wp, box, C, z, targets, y, radius, kind)[0]
        lm = adjoint.density_loss(wm, box, C, z, targets, y, radius, kind)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad.flat[c]) < rtol * np.abs(grad).max() + 1e-12, (c, fd, grad.flat[c])
