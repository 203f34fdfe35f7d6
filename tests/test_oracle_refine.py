"""Pins of the oracle's white-noise refinement (Appendix A).

What fixes it, independently of the code under test:
* Eq. A.1: every basis is orthonormal;
* the closed forms the paper prints for the child values (Eq. A.4 for one
  parent cell, Eq. A.15 for three child cells, Eqs. A.16-A.19 for four);
* a brute-force triple sum of Eq. A.14 / A.28 on single patches;
* the parent coefficients survive refinement and the new ones are the child
  grid's white noise (the reading stated in oracle/refine.py);
* refined white noise is again unit white noise (orthonormal maps of i.i.d.
  unit Gaussians);
* the comparison of the bases in the text around Fig. 6 (values in
  tests/golden/refine_fig6.txt).
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import noise
from oracle import refine as ref

KINDS = list(ref.KINDS)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "refine_fig6.txt")


@pytest.mark.parametrize("name,mat", [("two", ref.TWO_CELL), ("three", ref.THREE_CELL),
                                      ("four", ref.FOUR_CELL), ("four_linear", ref.FOUR_CELL_LINEAR),
                                      ("four_sine", ref.FOUR_CELL_SINE)])
def test_bases_orthonormal(name, mat):
    # Eq. A.1: sum_k E_i(k) E_j(k) = delta_ij
    n = mat.shape[0]
    for i in range(n):
        for j in range(n):
            s = sum(mat[i, k] * mat[j, k] for k in range(n))
            assert abs(s - (1.0 if i == j else 0.0)) < 1e-15, (name, i, j)


def test_first_two_functions_constant_and_odd():
    # E_0 constant; E_1 antisymmetric about the patch centre (no systematic shift)
    for mat in (ref.THREE_CELL, ref.FOUR_CELL, ref.FOUR_CELL_LINEAR, ref.FOUR_CELL_SINE):
        assert np.ptp(mat[0]) == 0.0
        assert np.allclose(mat[1], -mat[1][::-1], atol=0, rtol=0)


def test_hr_closed_form():
    # Eq. A.4: one parent value V and one new number R -> [(V - R)/sqrt2, (V + R)/sqrt2]
    v, r = 0.8125, -1.375
    got = ref.refine_1d([v], "hr", [r])
    want = [(v - r) / math.sqrt(2), (v + r) / math.sqrt(2)]
    assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_three_halves_closed_form():
    # Eq. A.15
    v0, v1, r = 1.25, -0.5, 0.75
    got = ref.refine_1d([v0, v1], "3/2", [r])
    s6 = math.sqrt(6)
    want = [(v0 + v1 - r) / s6 - (v1 - v0) / 2,
            (v0 + v1 + 2 * r) / s6,
            (v0 + v1 - r) / s6 + (v1 - v0) / 2]
    assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_doubling_closed_form():
    # Eqs. A.16-A.19
    v0, v1, r1, r2 = -0.3, 1.7, 0.4, -2.1
    got = ref.refine_1d([v0, v1], "2", [r1, r2])
    s8, s7, s2 = math.sqrt(8), math.sqrt(7), math.sqrt(2)
    d = (v1 - v0) / (4 * s2)
    want = [(v0 + v1) / s8 - s7 * d - r1 / 2 + r2 / 4,
            (v0 + v1) / s8 - d + r1 / 2 - s7 * r2 / 4,
            (v0 + v1) / s8 + d + r1 / 2 + s7 * r2 / 4,
            (v0 + v1) / s8 + s7 * d - r1 / 2 - r2 / 4]
    assert np.allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind", KINDS)
def test_single_patch_brute_force(kind):
    # Eqs. A.14 and A.28 written as explicit loops over one patch
    nl, nh, f, e = ref.KINDS[kind]
    rng = np.random.default_rng(5)
    parent = rng.standard_normal((nl, nl, nl))
    seed = 99
    child = ref.refine(parent, kind, seed)
    nc = nh  # the child box is one patch
    a = {}
    for i, j, k in itertools.product(range(nh), repeat=3):
        if i < nl and j < nl and k < nl:
            a[i, j, k] = sum(f[i, m] * f[j, q] * f[k, l] * parent[m, q, l]
                             for m, q, l in itertools.product(range(nl), repeat=3))
        else:
            a[i, j, k] = float(noise.noise_at(seed, [(i * nc + j) * nc + k])[0])
    for m, q, l in itertools.product(range(nh), repeat=3):
        want = sum(a[i, j, k] * e[i, m] * e[j, q] * e[k, l]
                   for i, j, k in itertools.product(range(nh), repeat=3))
        assert abs(child[m, q, l] - want) < 1e-13


@pytest.mark.parametrize("kind", KINDS)
def test_parent_coefficients_preserved(kind):
    nl, nh, f, _ = ref.KINDS[kind]
    n = 6 * nl
    parent = noise.white_noise(3, n)
    child = ref.refine(parent, kind, seed_child=11)
    a = ref.parent_coefficients(child, kind)
    # back to parent values with F^T (F orthonormal)
    back = np.einsum("im,jn,kl,xiyjzk->xmynzl", f, f, f, a).reshape(n, n, n)
    assert np.abs(back - parent).max() < 1e-13


@pytest.mark.parametrize("kind", ["2", "3/2", "4/3"])
def test_new_coefficients_are_child_noise(kind):
    nl, nh, _, e = ref.KINDS[kind]
    n = 4 * nl
    nc = n // nl * nh
    parent = noise.white_noise(8, n)
    child = ref.refine(parent, kind, seed_child=21)
    w = child.reshape(n // nl, nh, n // nl, nh, n // nl, nh)
    coef = np.einsum("im,jn,kl,xmynzl->xiyjzk", e, e, e, w)
    cn = noise.white_noise(21, nc).reshape(coef.shape)
    mask = np.ones((nh, nh, nh), dtype=bool)
    mask[:nl, :nl, :nl] = False
    for i, j, k in itertools.product(range(nh), repeat=3):
        if mask[i, j, k]:
            assert np.abs(coef[:, i, :, j, :, k] - cn[:, i, :, j, :, k]).max() < 1e-13


@pytest.mark.parametrize("kind", KINDS)
def test_sub_box_is_part_of_full_box(kind):
    nl, nh, _, _ = ref.KINDS[kind]
    n = 6 * nl
    parent = noise.white_noise(4, n)
    full = ref.refine(parent, kind, seed_child=5)
    origin, extent = (2 * nl, 4 * nl, 3 * nl), (2 * nl, 4 * nl, 5 * nl)  # wraps in y and z
    sub = ref.refine(parent, kind, 5, origin=origin, extent=extent)
    idx = [(o // nl * nh + np.arange(x // nl * nh)) % (n // nl * nh) for o, x in zip(origin, extent)]
    assert np.array_equal(sub, full[np.ix_(*idx)])


@pytest.mark.parametrize("kind", KINDS)
def test_refined_noise_is_white(kind):
    # child = orthonormal map of i.i.d. N(0,1) numbers -> i.i.d. N(0,1)
    n = 24  # a multiple of every parent patch
    child = ref.refine(noise.white_noise(17, n), kind, seed_child=18)
    c = child.ravel()
    m = c.size
    assert abs(c.mean()) < 5 / math.sqrt(m)
    assert abs(c.var() - 1) < 5 * math.sqrt(2 / m)
    for ax in range(3):
        r = np.mean(child * np.roll(child, 1, axis=ax))
        assert abs(r) < 5 / math.sqrt(m), ax


def _golden():
    vals = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                key, val = line.split()[:2]
                vals[key] = float(val)
    return vals


def test_fig6_basis_comparison():
    """1-D refinement of 1024-cell white noise by a factor 2 with each basis:
    mean amplitude of (refined - parent) at the parent's modes, relative to
    the basis of Eqs. A.10-A.13, as in the text around Fig. 6."""
    g = _golden()
    rng = np.random.default_rng(2024)
    m_real, nl_cells = 2000, 1024
    v = rng.standard_normal((m_real, nl_cells))
    vl = np.fft.rfft(v, axis=1)[:, : nl_cells // 2] / math.sqrt(nl_cells)

    def amp(kind):
        nl, nh, _, _ = ref.KINDS[kind]
        new = rng.standard_normal((m_real, nl_cells // nl, nh - nl))
        w = ref.refine_lines(v, kind, new)
        wh = np.fft.rfft(w, axis=1)[:, : nl_cells // 2] / math.sqrt(w.shape[1])
        return np.abs(wh - vl).mean(axis=0)[1:]

    a10, lin, hr, sine = amp("2"), amp("2-linear"), amp("hr"), amp("2-sine")
    hi = slice(nl_cells // 4, None)  # k / k_Ny > 0.5
    assert abs((lin / a10).mean() - g["linear_over_a10_mean"]) < 0.002
    assert abs((lin[hi] / a10[hi]).mean() - g["linear_over_a10_high_k"]) < 0.003
    assert abs((hr / a10).mean() - g["hr_over_a10_mean"]) < 0.01
    assert abs((sine / hr).mean() - g["sine_over_hr_mean"]) < 0.01
