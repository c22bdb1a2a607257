"""torch.autograd.Function over the library's hand-written discrete adjoint.

``burgers_velocity(theta0, nu, d, N, dx, dt, T)`` returns u(T), the coupled
Burgers' velocity recovered by the MRT-LB solver (Eq. (ui-compute)) after T
steps from theta0 (initialised with the fourth-order central-difference
gradient of theta0, so u depends on theta0 alone).  Its backward runs the
CUDA adjoint (reversed streaming, transposed collision, adjoint of the
recovery and of the initialisation) and returns dL/dtheta0 and dL/dnu; nu
enters through eps = nu dt / dx^2 and Theorem 2's relaxation set.  No
autograd tape is recorded through the solver: the kernels are the gradient.
"""

from __future__ import annotations

import torch

from . import lb


class _BurgersVelocity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta0, nu, d, N, dx, dt, T, precision, checkpoint):
        if theta0.dtype != torch.float64 or not theta0.is_cuda:
            raise TypeError("theta0 must be a float64 CUDA tensor")
        nu_v = float(nu.detach().item()) if isinstance(nu, torch.Tensor) else float(nu)
        want_nu = isinstance(nu, torch.Tensor) and nu.requires_grad
        solver = lb.Solver(d, N, nu_v, dx, dt, precision=precision)
        adj = lb.Adjoint(solver, T, checkpoint=checkpoint, want_nu=want_nu)
        u = adj.forward(theta0.contiguous())
        ctx.adj, ctx.solver, ctx.want_nu, ctx.nu_is_tensor = adj, solver, want_nu, isinstance(nu, torch.Tensor)
        if ctx.nu_is_tensor:
            ctx.nu_dtype, ctx.nu_device = nu.dtype, nu.device
        return u

    @staticmethod
    def backward(ctx, grad_u):
        adj = ctx.adj
        adj.seed(grad_u.contiguous().to(torch.float64))
        adj.step(adj.T)
        g0, dnu = adj.result()
        gnu = None
        if ctx.want_nu:
            gnu = torch.tensor(dnu, dtype=ctx.nu_dtype, device=ctx.nu_device)
        adj.close()
        ctx.solver.close()
        return g0, gnu, None, None, None, None, None, None, None


def burgers_velocity(theta0, nu, d, N, dx, dt, T, precision="fp64", checkpoint=0):
    """u(T) with gradients to theta0 (and to nu if it is a tensor requiring grad)."""
    return _BurgersVelocity.apply(theta0, nu, d, tuple(N), dx, dt, int(T), precision, int(checkpoint))
