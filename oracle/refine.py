"""White-noise resolution refinement of Appendix A (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Appendix A replaces every patch of N_L parent cells per axis by N_H child
cells. Inside a patch the values are expanded over orthonormal discrete bases
(Eq. A.1): F_i(m), m, i < N_L, for the parent and E_j(k), k, j < N_H, for the
child. The first N_L child coefficients equal the parent coefficients, the
other N_H - N_L are new unit Gaussian numbers, and the child values are
W(k) = sum_j a_j E_j(k) (Eq. A.14). In three dimensions the bases are tensor
products, E_ijk(m, n, l) = E_i(m) E_j(n) E_k(l) (Eq. A.28): a doubling turns
8 parent cells into 8 coefficients, adds 56 new ones and yields 64 values.

Bases (matrices B[i, m] = B_i(m)):
  hr         N_L = 1, N_H = 2: F_0 = [1], E of Eqs. A.2-A.3 (Hoffman-Ribak)
  3/2        N_L = 2, N_H = 3: F of Eqs. A.5-A.6, E of Eqs. A.7-A.9
  2          N_L = 2, N_H = 4: F of Eqs. A.5-A.6, E of Eqs. A.10-A.13
  2-linear   the same with E of Eqs. A.20-A.23
  2-sine     the same with E of Eqs. A.24-A.27
  4/3        N_L = 3, N_H = 4: F = the three-cell basis of Eqs. A.7-A.9,
             E of Eqs. A.10-A.13

Readings taken where Appendix A is silent:
* The 4/3 factor is named but its parent basis is not printed; the parent
  basis for three cells is taken to be the three-cell child basis of
  Eqs. A.7-A.9 (constant, linear, quadratic, as the appendix builds them).
* The appendix text calls the constant and linear parent functions F_1 and
  F_2 while the formulas number them F_0 and F_1; the formulas are followed.
* The new coefficients are drawn from the white noise of the child grid
  (the Philox / Box-Muller field of ``noise``, with its own seed) at the
  child cell that has the coefficient's position in the patch: coefficient
  (i, j, k) of the patch whose first child cell is (X, Y, Z) takes the noise
  value of child cell (X + i, Y + j, Z + k) of the full refined grid. So the
  result does not depend on how the work is split, and a refined sub-box is
  exactly that part of the refined full box.
* Patches tile the box from the origin; a sub-box starts on a patch boundary
  and the parent grid is periodic.

Pinned in tests/test_oracle_refine.py: Eq. A.1 for every basis, the closed
forms Eqs. A.4, A.15 and A.16-A.19, the preservation of the parent
coefficients, the variance of the child field, and the comparison of the
bases in the text around Fig. 6 (values in tests/golden/refine_fig6.txt).
"""
import numpy as np

from .noise import noise_at

_R2, _R3, _R6, _R7, _R20 = np.sqrt(2.0), np.sqrt(3.0), np.sqrt(6.0), np.sqrt(7.0), np.sqrt(20.0)

# Eqs. A.2-A.3: one parent cell refined into two (also Eqs. A.5-A.6 for two
# parent cells).
TWO_CELL = np.array([[1 / _R2, 1 / _R2],
                     [-1 / _R2, 1 / _R2]])
# Eqs. A.7-A.9: three cells.
THREE_CELL = np.array([[1 / _R3, 1 / _R3, 1 / _R3],
                       [-1 / _R2, 0.0, 1 / _R2],
                       [-1 / _R6, 2 / _R6, -1 / _R6]])
# Eqs. A.10-A.13: four cells, the paper's choice.
FOUR_CELL = np.array([[0.5, 0.5, 0.5, 0.5],
                      [-_R7 / 4, -0.25, 0.25, _R7 / 4],
                      [-0.5, 0.5, 0.5, -0.5],
                      [0.25, -_R7 / 4, _R7 / 4, -0.25]])
# Eqs. A.20-A.23: four cells with E_1 linear in k.
FOUR_CELL_LINEAR = np.array([[0.5, 0.5, 0.5, 0.5],
                             [-3 / _R20, -1 / _R20, 1 / _R20, 3 / _R20],
                             [-0.5, 0.5, 0.5, -0.5],
                             [1 / _R20, -3 / _R20, 3 / _R20, -1 / _R20]])
# Eqs. A.24-A.27: four cells with E_1 a sampled sine of the patch period.
FOUR_CELL_SINE = np.array([[0.5, 0.5, 0.5, 0.5],
                           [-0.5, -0.5, 0.5, 0.5],
                           [-0.5, 0.5, 0.5, -0.5],
                           [0.5, -0.5, 0.5, -0.5]])

# kind -> (N_L, N_H, F, E)
KINDS = {
    "hr": (1, 2, np.array([[1.0]]), TWO_CELL),
    "3/2": (2, 3, TWO_CELL, THREE_CELL),
    "2": (2, 4, TWO_CELL, FOUR_CELL),
    "2-linear": (2, 4, TWO_CELL, FOUR_CELL_LINEAR),
    "2-sine": (2, 4, TWO_CELL, FOUR_CELL_SINE),
    "4/3": (3, 4, THREE_CELL, FOUR_CELL),
}


def refine_1d(parent, kind, new):
    """One patch in one dimension: N_L parent values and N_H - N_L new
    coefficients -> N_H child values (Eq. A.14 with a_i = sum_m F_i(m) V_m)."""
    nl, nh, f, e = KINDS[kind]
    a = np.concatenate([f @ np.asarray(parent, dtype=np.float64),
                        np.asarray(new, dtype=np.float64)])
    assert a.shape == (nh,)
    return a @ e


def refine_lines(parent, kind, new):
    """Many 1-D lines at once: parent (M, n), new (M, n / N_L, N_H - N_L)
    -> (M, n N_H / N_L). Patches tile each line from index 0."""
    nl, nh, f, e = KINDS[kind]
    p = np.asarray(parent, dtype=np.float64)
    m, n = p.shape
    a = np.empty((m, n // nl, nh))
    a[:, :, :nl] = p.reshape(m, n // nl, nl) @ f.T
    a[:, :, nl:] = new
    return (a @ e).reshape(m, n // nl * nh)


def child_size(n, kind):
    nl, nh, _, _ = KINDS[kind]
    if n % nl:
        raise ValueError("grid size not a multiple of the parent patch")
    return n // nl * nh


def refine_patches(v, kind, seed_child, n, gp):
    """Child values of a list of patches (Eqs. A.14, A.28).

    ``v``: (P, N_L, N_L, N_L) parent values of each patch; ``gp``: (P, 3)
    patch coordinates in the whole grid (patch (X, Y, Z) holds parent cells
    N_L X .. N_L X + N_L - 1 per axis); ``n``: parent points per axis.
    Returns (P, N_H, N_H, N_H)."""
    nl, nh, f, e = KINDS[kind]
    nc = child_size(n, kind)
    v = np.asarray(v, dtype=np.float64).reshape(-1, nl, nl, nl)
    gp = np.asarray(gp, dtype=np.int64).reshape(-1, 3)
    # every coefficient position takes the child noise at its child cell ...
    k = np.arange(nh)
    cx = gp[:, 0, None] * nh + k  # (P, N_H) child coordinates per axis
    cy = gp[:, 1, None] * nh + k
    cz = gp[:, 2, None] * nh + k
    idx = (cx[:, :, None, None] * nc + cy[:, None, :, None]) * nc + cz[:, None, None, :]
    a = noise_at(seed_child, idx.ravel()).reshape(-1, nh, nh, nh)
    # ... except the first N_L^3: a_ijk = sum_mnl F_i(m) F_j(n) F_k(l) V(m, n, l)
    a[:, :nl, :nl, :nl] = np.einsum("im,jn,kl,pmnl->pijk", f, f, f, v)
    # W(m, n, l) = sum_ijk a_ijk E_i(m) E_j(n) E_k(l)
    return np.einsum("im,jn,kl,pijk->pmnl", e, e, e, a)


def refine(parent, kind, seed_child, origin=(0, 0, 0), extent=None):
    """Refined white noise of the sub-box [origin, origin + extent) (parent
    cells, periodic) of the parent grid; returns the child grid of
    extent * N_H / N_L cells per axis."""
    parent = np.asarray(parent, dtype=np.float64)
    n = parent.shape[0]
    nl, nh, _, _ = KINDS[kind]
    child_size(n, kind)
    if extent is None:
        extent = (n, n, n)
    for o, x in zip(origin, extent):
        if o % nl or x % nl or not 0 < x <= n or not 0 <= o < n:
            raise ValueError("origin / extent must be multiples of the parent patch inside the box")
    npx, npy, npz = (x // nl for x in extent)
    # patch coordinates in the whole grid (periodic), x slowest
    gx, gy, gz = ((o // nl + np.arange(x // nl)) % (n // nl) for o, x in zip(origin, extent))
    gp = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), axis=-1).reshape(-1, 3)
    # parent values of each patch
    off = np.arange(nl)
    px = gp[:, 0, None] * nl + off
    py = gp[:, 1, None] * nl + off
    pz = gp[:, 2, None] * nl + off
    v = parent[px[:, :, None, None], py[:, None, :, None], pz[:, None, None, :]]
    w = refine_patches(v, kind, seed_child, n, gp)
    # patches back into the child box
    return (w.reshape(npx, npy, npz, nh, nh, nh).transpose(0, 3, 1, 4, 2, 5)
            .reshape(npx * nh, npy * nh, npz * nh))


def parent_coefficients(child, kind):
    """Projection of a child grid on the first N_L^3 tensor basis functions
    of each patch: (P, N_L, P, N_L, P, N_L) coefficients."""
    nl, nh, _, e = KINDS[kind]
    c = np.asarray(child, dtype=np.float64)
    px, py, pz = (s // nh for s in c.shape)
    w = c.reshape(px, nh, py, nh, pz, nh)
    el = e[:nl]
    return np.einsum("im,jn,kl,xmynzl->xiyjzk", el, el, el, w)
