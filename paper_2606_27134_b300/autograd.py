"""torch.autograd.Function around dmk_eval.

u_t = sum_s sum*_p K(x_t - x_s + p) rho_s.  For L = sum_t g_t . u_t and an even kernel whose
matrix is symmetric (Laplace, Stokeslet: K(-x) = K(x), K_jl = K_lj), the sum is self-adjoint:
    dL/drho_s = sum_t K(x_t - x_s)^T g_t = v(x_s),         v = the same sum with strengths g;
    dL/dx_a   = sum_j g_a,j grad u_j(x_a) + sum_l rho_a,l grad v_l(x_a),
so the backward pass is one more evaluation of the same hot path (every stage: leaf residual
sums, plane waves, root Fourier sum) with strengths g and target gradients.  The forward saves
the field gradient of u.  Both passes run in the CUDA library.
"""
import torch

from . import dmk

SELF_ADJOINT = ("laplace", "stokeslet")


class _DMKFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, strengths, plan):
        need_grad = points.requires_grad or strengths.requires_grad
        u, gu = plan.eval(points.detach(), strengths.detach(), grad=need_grad)
        ctx.plan = plan
        ctx.save_for_backward(points, strengths, gu if need_grad else torch.empty(0, device=points.device))
        return u

    @staticmethod
    def backward(ctx, g):
        points, strengths, gu = ctx.saved_tensors
        plan = ctx.plan
        N = points.shape[0]
        g = g.contiguous().reshape(N, plan.d_u)
        v, gv = plan.eval(points.detach(), g.to(torch.float64), grad=True)
        d_rho = v.reshape(strengths.shape) if ctx.needs_input_grad[1] else None
        d_x = None
        if ctx.needs_input_grad[0]:
            rho = strengths.reshape(N, plan.d_rho)
            d_x = torch.einsum("tij,tj->ti", gu, g) + torch.einsum("tij,tj->ti", gv, rho)
        return d_x, d_rho, None


class Potential(torch.nn.Module):
    """u = Potential(kernel, D, L, tol)(points, strengths), differentiable in both arguments.

    Supported for the self-adjoint kernels (Laplace, Stokeslet).  Points and strengths are CUDA
    float64 tensors of shapes (N, 3) and (N, d_rho).
    """

    def __init__(self, kernel, D, L, tol, precision="mixed", n_s=250, stream=None):
        super().__init__()
        if kernel not in SELF_ADJOINT:
            raise NotImplementedError("autograd wrapper covers the self-adjoint kernels " + str(SELF_ADJOINT))
        self.plan = dmk.Plan(kernel, D, L, tol, precision=precision, n_s=n_s, stream=stream)

    def forward(self, points, strengths):
        return _DMKFunction.apply(points, strengths, self.plan)


def energy_and_forces(points, charges, D, L, tol, precision="mixed", n_s=250):
    """Laplace electrostatic energy E = 1/2 sum_t q_t u_t and forces F = -dE/dx through autograd."""
    pot = Potential("laplace", D, L, tol, precision=precision, n_s=n_s)
    x = points.detach().clone().requires_grad_(True)
    u = pot(x, charges.reshape(-1, 1))
    E = 0.5 * (charges.reshape(-1) * u.reshape(-1)).sum()
    (gx,) = torch.autograd.grad(E, x)
    return E.detach(), -gx
