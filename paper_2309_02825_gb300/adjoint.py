"""torch.autograd.Function over the library's hand-written discrete adjoint.

``burgers_velocity(theta0, nu, d, N, dx, dt, T)`` returns u(T), the coupled
Burgers' velocity recovered by the MRT-LB solver (Eq. (ui-compute)) after T
steps from theta0 (initialised with the fourth-order central-difference
gradient of theta0, so u depends on theta0 alone); ``burgers_fields`` returns
(u(T), theta(T)).  Their backward runs the CUDA adjoint (reversed streaming,
transposed collision, adjoint of the recovery and of the initialisation)
and returns dL/dtheta0 and dL/dnu; nu enters through eps = nu dt / dx^2 and
Theorem 2's relaxation set.  No autograd tape is recorded through the
solver: the kernels are the gradient.

Device memory: one solver context and one adjoint workspace (checkpoints,
adjoint fields) per (device, d, N, dx, dt, T, precision, checkpoint
interval, dL/dnu wanted), created on first use and reused by every later
call with the same key, so a training loop allocates them once.  The
viscosity is set in place (lb_set_viscosity).  A workspace holds the forward
states of the last forward that ran in it; a backward whose forward was
overwritten since (a second call with the same key in one graph, or
``retain_graph`` after another forward) first re-runs its own forward from
the saved theta0 and nu, so gradients are always those of the node's own
inputs.  ``clear_cache()`` releases the workspaces.
"""

from __future__ import annotations

import itertools
from collections import OrderedDict

import torch

from . import lb

_MAX_CACHED = 4
_cache: "OrderedDict[tuple, _Workspace]" = OrderedDict()
_tokens = itertools.count(1)
stats = {"workspaces_created": 0, "forward_replays": 0}


class _Workspace:
    def __init__(self, d, N, nu, dx, dt, T, precision, checkpoint, want_nu):
        self.solver = lb.Solver(d, N, nu, dx, dt, precision=precision)
        self.adj = lb.Adjoint(self.solver, T, checkpoint=checkpoint, want_nu=want_nu)
        self.nu = float(nu)
        self.owner = 0  # token of the forward whose states the workspace holds
        stats["workspaces_created"] += 1

    def run_forward(self, theta0, nu, token):
        if nu != self.nu:
            self.solver.set_viscosity(nu)
            self.nu = nu
        th = torch.empty(self.solver.shape, dtype=torch.float64, device=theta0.device)
        u = self.adj.forward(theta0, theta=th)
        self.owner = token
        return u, th

    def close(self):
        self.adj.close()
        self.solver.close()
        self.closed = True

    closed = False


def _workspace(key, nu):
    ws = _cache.get(key)
    if ws is None:
        _, d, N, dx, dt, T, precision, checkpoint, want_nu = key
        ws = _Workspace(d, N, nu, dx, dt, T, precision, checkpoint, want_nu)
        _cache[key] = ws
        while len(_cache) > _MAX_CACHED:
            _, old = _cache.popitem(last=False)
            old.close()
    else:
        _cache.move_to_end(key)
    return ws


def clear_cache():
    """Release every cached solver and adjoint workspace."""
    while _cache:
        _, ws = _cache.popitem()
        ws.close()


class _BurgersFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta0, nu, d, N, dx, dt, T, precision, checkpoint):
        if theta0.dtype != torch.float64 or not theta0.is_cuda:
            raise TypeError("theta0 must be a float64 CUDA tensor")
        nu_v = float(nu.detach().item()) if isinstance(nu, torch.Tensor) else float(nu)
        want_nu = isinstance(nu, torch.Tensor) and nu.requires_grad
        key = (theta0.device.index, d, tuple(N), dx, dt, T, precision, checkpoint, want_nu)
        theta0 = theta0.detach().contiguous()
        with torch.cuda.device(theta0.device):
            ws = _workspace(key, nu_v)
            token = next(_tokens)
            u, th = ws.run_forward(theta0, nu_v, token)
        ctx.ws, ctx.key, ctx.token, ctx.nu_v, ctx.want_nu = ws, key, token, nu_v, want_nu
        ctx.nu_is_tensor = isinstance(nu, torch.Tensor)
        if ctx.nu_is_tensor:
            ctx.nu_dtype, ctx.nu_device = nu.dtype, nu.device
        ctx.save_for_backward(theta0)
        ctx.set_materialize_grads(False)
        return u, th

    @staticmethod
    def backward(ctx, grad_u, grad_theta):
        (theta0,) = ctx.saved_tensors
        ws = ctx.ws
        if grad_u is None and grad_theta is None:
            return (None,) * 9
        with torch.cuda.device(theta0.device):
            if ws.closed:  # released since (cache eviction or clear_cache): take a live one
                ws = ctx.ws = _workspace(ctx.key, ctx.nu_v)
            if ws.owner != ctx.token:  # another forward ran in this workspace since
                ws.run_forward(theta0, ctx.nu_v, ctx.token)
                stats["forward_replays"] += 1
            gu = None if grad_u is None else grad_u.detach().to(torch.float64).contiguous()
            gt = None if grad_theta is None else grad_theta.detach().to(torch.float64).contiguous()
            ws.adj.seed(gu, gt)
            ws.adj.step(ws.adj.T)
            g0, dnu = ws.adj.result()
        gnu = None
        if ctx.want_nu:
            gnu = torch.tensor(dnu, dtype=ctx.nu_dtype, device=ctx.nu_device)
        return g0, gnu, None, None, None, None, None, None, None


def burgers_fields(theta0, nu, d, N, dx, dt, T, precision="fp64", checkpoint=0):
    """(u(T), theta(T)) with gradients to theta0 (and to nu if it is a tensor
    requiring grad) of any loss of u(T) and theta(T)."""
    return _BurgersFields.apply(theta0, nu, int(d), tuple(int(n) for n in N), float(dx), float(dt), int(T),
                                precision, int(checkpoint))


def burgers_velocity(theta0, nu, d, N, dx, dt, T, precision="fp64", checkpoint=0):
    """u(T) with gradients to theta0 (and to nu if it is a tensor requiring grad)."""
    return burgers_fields(theta0, nu, d, N, dx, dt, T, precision, checkpoint)[0]
