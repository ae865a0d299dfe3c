"""torch.autograd.Function around dmk_eval and dmk_vjp.

u_t = sum_s sum*_p K(x_t - x_s + p) rho_s.  For L = sum_t g_t . u_t and a kernel with
K(-x) = K(x)^T (Laplace, Stokeslet: even and symmetric; rotlet: odd and antisymmetric), the
sum is self-adjoint:
    dL/drho_s = sum_t K(x_t - x_s)^T g_t = v(x_s),         v = the same sum with strengths g;
    dL/dx_a   = sum_j g_a,j grad u_j(x_a) + sum_l rho_a,l grad v_l(x_a),
so the backward pass is one more evaluation of the same hot path (every stage: leaf residual
sums, plane waves, root Fourier sum) with strengths g and target gradients, followed by the
assembly of dL/dx; dmk_vjp does all of it in the CUDA library.  The forward saves the field
gradient of u.  The stresslet (9 strength components, 3 outputs) is not self-adjoint; its
kernel is fully symmetric in its three indices and odd, so dmk_vjp uses three evaluations with
the strengths g (x) e_m instead.
"""
import torch

from . import dmk

SELF_ADJOINT = ("laplace", "stokeslet", "rotlet")
DIFFERENTIABLE = SELF_ADJOINT + ("stresslet",)


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
        want_x, want_rho = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        d_rho, d_x = plan.vjp(points.detach(), strengths.detach(), gu, g.to(torch.float64),
                              want_strengths=want_rho, want_points=want_x)
        if d_rho is not None:
            d_rho = d_rho.reshape(strengths.shape)
        return d_x, d_rho, None


class Potential(torch.nn.Module):
    """u = Potential(kernel, D, L, tol)(points, strengths), differentiable in both arguments.

    Supported for every kernel (the stresslet through its symmetric form).  Points and strengths
    are CUDA float64 tensors of shapes (N, 3) and (N, d_rho).  Laplace with D = 1 or 2 needs
    neutral strengths in the forward pass (Sec. 5.2); the upstream gradient of the backward pass
    need not be neutral: dL/dpoints is exact and dL/dstrengths is exact up to an additive
    constant, which no neutral change of the strengths sees.
    """

    def __init__(self, kernel, D, L, tol, precision="mixed", n_s=250, stream=None):
        super().__init__()
        if kernel not in DIFFERENTIABLE:
            raise NotImplementedError("autograd wrapper covers the kernels " + str(DIFFERENTIABLE))
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
