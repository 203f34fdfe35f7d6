"""Differentiable density of the Zel'dovich particles and its adjoint (oracle).

Test infrastructure for the adjoint form (gradients of a loss on the smoothed
particle density with respect to the white noise W). The paper has no such
form; the forward map W -> psi is that of Eqs. 1-2 (``fields.zeldovich``).
Readings taken:

* Density: one particle per Lagrangian cell at x = q + psi (Eq. 3 positions,
  periodic); cloud-in-cell assignment to nodes at the cell centres with
  linear weights per axis; delta = (particles per node) - 1.
* Smoothing: Gaussian exp(-k^2 R^2 / 2) on the periodic grid, the modes with
  any |m_j| = N/2 dropped (as in the forward path).
* Loss: L = sum_t (delta_s(c_t) - y_t)^2 over target cells c_t.
* Linear alternative: delta = -div psi (the Gaussian field of Eq. 1), which
  makes the loss exactly quadratic in W.

The transposes are written out from the definitions: the CIC adjoint is the
gradient of the weights; the smoothing is symmetric; the map W -> psi_j,
J_j = F^-1 diag(i m_j U) F with a purely imaginary Hermitian multiplier, has
J_j^T = -J_j. Pinned in tests/test_oracle_adjoint.py by dot-product tests and
central finite differences.
"""
import numpy as np

from . import fields


def _grid_coords(n):
    i = np.arange(n, dtype=np.float64)
    return (i[:, None, None], i[None, :, None], i[None, None, :])


def _cic_geometry(psi, box, q_offset):
    n = psi[0].shape[0]
    cell = box / n
    base = _grid_coords(n)
    i0, frac = [], []
    for j in range(3):
        u = base[j] + (q_offset - 0.5) + psi[j] / cell
        fl = np.floor(u)
        i0.append(np.mod(fl, n).astype(np.int64))
        frac.append(u - fl)
    return n, cell, i0, frac


def cic_density(psi, box, q_offset=0.5):
    """delta(c) = sum_p w_c(x_p) - 1 with CIC weights (nodes at cell centres)."""
    n, _, i0, frac = _cic_geometry(psi, box, q_offset)
    delta = np.full(n ** 3, -1.0)
    for corner in range(8):
        hi = [(corner >> (2 - j)) & 1 for j in range(3)]
        w = np.ones((n, n, n))
        idx = np.zeros((n, n, n), dtype=np.int64)
        for j in range(3):
            w = w * (frac[j] if hi[j] else 1.0 - frac[j])
            idx = idx * n + np.mod(i0[j] + hi[j], n)
        np.add.at(delta, idx.ravel(), w.ravel())
    return delta.reshape(n, n, n)


def cic_adjoint(psi, g, box, q_offset=0.5):
    """g_psi_j(p) = sum_c g(c) dw_c(x_p)/dpsi_j (the transpose of the CIC Jacobian)."""
    n, cell, i0, frac = _cic_geometry(psi, box, q_offset)
    gf = g.ravel()
    out = [np.zeros((n, n, n)) for _ in range(3)]
    for corner in range(8):
        hi = [(corner >> (2 - j)) & 1 for j in range(3)]
        w = [frac[j] if hi[j] else 1.0 - frac[j] for j in range(3)]
        dw = [1.0 if hi[j] else -1.0 for j in range(3)]
        idx = np.zeros((n, n, n), dtype=np.int64)
        for j in range(3):
            idx = idx * n + np.mod(i0[j] + hi[j], n)
        gv = gf[idx]
        out[0] += gv * dw[0] * w[1] * w[2]
        out[1] += gv * w[0] * dw[1] * w[2]
        out[2] += gv * w[0] * w[1] * dw[2]
    return [o / cell for o in out]


def smooth(field, box, radius):
    """F^-1[exp(-k^2 R^2/2) F field], Nyquist modes dropped."""
    n = field.shape[0]
    fk = np.fft.rfftn(field)
    mx, my, mz = fields.integer_modes(n)
    k2 = (2 * np.pi / box) ** 2 * (mx * mx + my * my + mz * mz).astype(np.float64)
    keep = (np.abs(mx) != n // 2) & (np.abs(my) != n // 2) & (mz != n // 2)
    g = np.where(keep, np.exp(-0.5 * k2 * radius * radius), 0.0)
    return np.fft.irfftn(fk * g, s=field.shape, axes=(0, 1, 2))


def psi_map(w, box, cosmo, z_init, j):
    """psi_j as a linear function of the noise grid w (Eqs. 1-2)."""
    n = w.shape[0]
    return fields.zeldovich(n, box, cosmo, z_init, noise=w, components=(j,))["psi"][j]


def psi_adjoint(g_psi, box, cosmo, z_init):
    """sum_j J_j^T g_j with J_j^T = -J_j (imaginary Hermitian multiplier)."""
    out = None
    for j in range(3):
        if g_psi[j] is None:
            continue
        term = -psi_map(np.asarray(g_psi[j], dtype=np.float64), box, cosmo, z_init, j)
        out = term if out is None else out + term
    return out


def linear_density(w, box, cosmo, z_init):
    """delta = -div psi: the Gaussian field of Eq. 1 (symmetric in w)."""
    n = w.shape[0]
    return fields.zeldovich(n, box, cosmo, z_init, noise=w, want_delta=True, components=())["delta"]


def density_loss(w, box, cosmo, z_init, targets, y, radius, kind="cic"):
    """L = sum_t (delta_s(c_t) - y_t)^2 and the intermediates."""
    if kind == "cic":
        psi = [psi_map(w, box, cosmo, z_init, j) for j in range(3)]
        d = cic_density(psi, box)
    else:
        psi = None
        d = linear_density(w, box, cosmo, z_init)
    ds = smooth(d, box, radius)
    r = ds.ravel()[targets] - y
    return float(np.sum(r * r)), psi, ds


def density_loss_grad(w, box, cosmo, z_init, targets, y, radius, kind="cic"):
    """dL/dW by the adjoint chain: scatter -> smooth -> CIC adjoint -> psi adjoint."""
    _, psi, ds = density_loss(w, box, cosmo, z_init, targets, y, radius, kind)
    g_s = np.zeros(ds.size)
    np.add.at(g_s, targets, 2.0 * (ds.ravel()[targets] - y))
    g_d = smooth(g_s.reshape(ds.shape), box, radius)
    if kind == "cic":
        g_psi = cic_adjoint(psi, g_d, box)
        return psi_adjoint(g_psi, box, cosmo, z_init)
    return linear_density(g_d, box, cosmo, z_init)
