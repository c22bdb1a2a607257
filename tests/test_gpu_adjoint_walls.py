"""GPU discrete adjoint on grids with mirror walls, against the oracle's wall
model (the periodic FP64 oracle on the grid doubled by even reflection).

dL/dtheta0 is checked against the exact dense Jacobian: theta0 -> f_T is
linear (initialisation with the reflected fourth-order gradient, then T
linear steps), so its columns are oracle runs of unit vectors, and
u = (2 - s1) c J / theta is differentiated by hand.  dL/dnu is checked
against the complex-step derivative of the same wall model (the complex
forward map of the oracle tests, on the evenly doubled grid, restricted to
the grid's nodes), whose real part must reproduce the oracle's loss.  The
loss is L = 1/2 sum over the grid's nodes of |u(T) - u_target|^2.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W
from tests.test_oracle_adjoint import complex_forward_u

pytestmark = pytest.mark.gpu


def _case(d, N, seed):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 4, 2, 0.05, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2048 * dx * dx / nu
    rng = np.random.default_rng(seed + 1)
    ut = 0.01 * rng.standard_normal((d,) + tuple(reversed(N)))
    return prob.theta(N, dx), ut, nu, dx, dt


def _oracle_u_parts(m, th0, T):
    """theta and J on the grid's nodes after T steps, from the doubled grid."""
    f = m.run(m.initialize(th0), T)
    e = m.full.matrices()["e"]
    d = m.d
    th = f.sum(axis=0)
    J = np.stack([np.tensordot(e[:, a], f, axes=(0, 0)) for a in range(d)])
    return O.restrict(th, d, m.N), O.restrict(J, d, m.N, vector=True)


def _oracle_loss(d, N, mirror, nu, dx, dt, th0, ut, T):
    m = O.MirrorModel(d, N, mirror, nu, dx, dt)
    _, _, u = m.recover(m.run(m.initialize(th0), T))
    return 0.5 * float(np.sum((u - ut) ** 2))


def _complex_step_dnu(d, N, mirror, nu, dx, dt, th0, ut, T):
    """(L, dL/dnu) of the wall model by the complex step h = 1e-20 nu."""
    h = 1e-20 * nu
    full = O.even_extension(th0, d, mirror)
    Nf = tuple(reversed(full.shape))
    u = O.restrict(complex_forward_u(d, Nf, nu + 1j * h, dx, dt, full, T), d, N, vector=True)
    L = 0.5 * np.sum((u - ut) ** 2)
    return L.real, L.imag / h


def _dense_gradient(d, N, mirror, nu, dx, dt, th0, ut, T):
    m = O.MirrorModel(d, N, mirror, nu, dx, dt)
    p = m.params
    ucoef = (2.0 - p["s1"]) * p["c"]
    th, J = _oracle_u_parts(m, th0, T)
    r = ucoef * J / th[None] - ut
    g = np.zeros(th0.size)
    for j in range(th0.size):
        ej = np.zeros(th0.size)
        ej[j] = 1.0
        dth, dJ = _oracle_u_parts(m, ej.reshape(th0.shape), T)
        du = ucoef * (dJ * th[None] - J * dth[None]) / (th[None] ** 2)
        g[j] = np.sum(r * du)
    return g.reshape(th0.shape)


def _gpu_gradient(d, N, mirror, nu, dx, dt, th0, ut, T, precision):
    kinds = ["mirror" if w else "periodic" for w in mirror]
    s = lb.Solver(d, N, nu, dx, dt, precision=precision, theta_ref=1.5, boundary=kinds)
    a = lb.Adjoint(s, T, want_nu=True)
    u = a.forward(torch.from_numpy(th0).cuda())
    a.seed((u - torch.from_numpy(ut).cuda()).contiguous())
    a.step(T)
    g, dnu = a.result()
    g = g.cpu().numpy()
    a.close()
    s.close()
    return g, dnu


CASES = [(1, (9,), (True,), 7), (2, (7, 6), (True, False), 5), (2, (6, 5), (True, True), 6),
         (3, (5, 4, 4), (True, False, True), 4), (3, (4, 5, 3), (True, True, True), 3)]


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("d,N,mirror,T", CASES)
def test_wall_adjoint_matches_dense_jacobian_and_nu_differences(d, N, mirror, T, precision):
    th0, ut, nu, dx, dt = _case(d, N, 90 + d)
    g_ref = _dense_gradient(d, N, mirror, nu, dx, dt, th0, ut, T)
    g, dnu = _gpu_gradient(d, N, mirror, nu, dx, dt, th0, ut, T, precision)
    rel = np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))
    L_cs, dnu_cs = _complex_step_dnu(d, N, mirror, nu, dx, dt, th0, ut, T)
    assert L_cs == pytest.approx(_oracle_loss(d, N, mirror, nu, dx, dt, th0, ut, T), rel=1e-13)
    print("wall adjoint %s d=%d N=%s walls=%s: dtheta0 rel %.2e, dnu rel %.2e"
          % (precision, d, N, mirror, rel, abs(dnu / dnu_cs - 1)))
    assert rel <= 1e-12
    assert dnu == pytest.approx(dnu_cs, rel=1e-12)


def test_wall_adjoint_fp32_shifted_tracks_fp64():
    d, N, mirror, T = 2, (40, 30), (True, True), 20
    th0, ut, nu, dx, dt = _case(d, N, 7)
    g64, dnu64 = _gpu_gradient(d, N, mirror, nu, dx, dt, th0, ut, T, "fp64")
    g32, dnu32 = _gpu_gradient(d, N, mirror, nu, dx, dt, th0, ut, T, "fp32s")
    assert np.max(np.abs(g32 - g64)) <= 1e-3 * np.max(np.abs(g64))
    assert dnu32 == pytest.approx(dnu64, rel=1e-3)


def test_wall_change_after_forward_is_refused():
    """Checkpoints belong to the geometry of the forward pass: reverse steps
    after lb_set_boundary report LB_ESTATE until a new forward."""
    d, N, T = 2, (12, 10), 6
    th0, ut, nu, dx, dt = _case(d, N, 5)
    s = lb.Solver(d, N, nu, dx, dt, precision="fp64", theta_ref=1.5, boundary=["mirror", "periodic"])
    a = lb.Adjoint(s, T, want_nu=True)
    u = a.forward(torch.from_numpy(th0).cuda())
    a.seed((u - torch.from_numpy(ut).cuda()).contiguous())
    a.step(2)
    lb.lb_set_boundary(s.ctx, ["periodic", "periodic"])
    with pytest.raises(lb.LBError) as ei:
        a.step(1)
    assert ei.value.status == lb.LB_ESTATE
    u = a.forward(torch.from_numpy(th0).cuda())  # a new forward on the new geometry
    a.seed((u - torch.from_numpy(ut).cuda()).contiguous())
    a.step(T)
    g, dnu = a.result()
    assert bool(torch.isfinite(g).all()) and np.isfinite(dnu)
    a.close()
    s.close()
