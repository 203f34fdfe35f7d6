"""Differentiable pieces of the initial-conditions path for gradient-based
fitting of constrained realizations (torch.autograd.Function wrappers).

Every forward and backward runs in the library's kernels:

* ``ZeldovichPsi``   noise W -> displacements psi_j (Eqs. 1-2); backward is the
                     transpose g_W = sum_j J_j^T g_j = -sum_j J_j g_j, computed
                     by re-running the transform chain on the gradients (no
                     transform intermediates are stored).
* ``CicDensity``     psi -> CIC density contrast of the particles at q + psi;
                     backward gathers the weight derivatives at psi.
* ``GaussianSmooth`` field -> exp(-k^2 R^2/2)-smoothed field (symmetric: the
                     backward is the same smoothing).
* ``LinearDensity``  noise -> delta of Eq. 1 (= -div psi); symmetric, so the
                     backward is the same map applied to the gradient.

``smoothed_density_loss`` composes them into L = sum_t (delta_s(c_t) - y_t)^2;
the gather at the target cells and the square are the caller's objective.
"""
import torch


class ZeldovichPsi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, noise, plan):
        ctx.plan = plan
        out = plan.zeldovich(noise=noise.contiguous(), psi=True, pos=False, vel=False)
        return tuple(out["psi"])

    @staticmethod
    def backward(ctx, g0, g1, g2):
        gs = [None if g is None else g.contiguous() for g in (g0, g1, g2)]
        if all(g is None for g in gs):
            return None, None
        return ctx.plan.zeldovich_adjoint(gs), None


class CicDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi_x, psi_y, psi_z, plan):
        ctx.plan = plan
        ctx.save_for_backward(psi_x, psi_y, psi_z)
        return plan.cic_density([psi_x.contiguous(), psi_y.contiguous(), psi_z.contiguous()])

    @staticmethod
    def backward(ctx, g):
        psi = [t.contiguous() for t in ctx.saved_tensors]
        gx, gy, gz = ctx.plan.cic_density_adjoint(psi, g.contiguous())
        return gx, gy, gz, None


class GaussianSmooth(torch.autograd.Function):
    @staticmethod
    def forward(ctx, field, plan, radius):
        ctx.plan, ctx.radius = plan, radius
        return plan.smooth(field.contiguous(), radius)

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.smooth(g.contiguous(), ctx.radius), None, None


class LinearDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, noise, plan):
        ctx.plan = plan
        return plan.gaussian_field(noise=noise.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.gaussian_field(noise=g.contiguous()), None


def smoothed_density_loss(noise, plan, targets, y, radius=8.0, density="cic"):
    """L = sum_t (delta_s(c_t) - y_t)^2 with delta_s the Gaussian-smoothed CIC
    (or linear) density of the Zel'dovich particles made from ``noise``.

    ``targets``: int64 tensor of flat cell indices; ``y``: target values."""
    if density == "cic":
        psi = ZeldovichPsi.apply(noise, plan)
        delta = CicDensity.apply(psi[0], psi[1], psi[2], plan)
    else:
        delta = LinearDensity.apply(noise, plan)
    ds = GaussianSmooth.apply(delta, plan, radius)
    r = ds.reshape(-1)[targets] - y
    return (r * r).sum()
