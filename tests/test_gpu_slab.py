"""Slab decomposition on one GPU: P parts of one periodic grid, each a
separate context, with the ghost layers refreshed before every sweep by
device copies routed as between processes (part p's "up" buffer to p+1's
lower ghost layer, its "down" buffer to p-1's upper ghost layer, periodic).
The owned layers must equal the single-grid solve bit for bit (same
arithmetic on the same inputs) and the oracle to the FP64 bar."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import slab as SL
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(d, N):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.1, 1.5, 30 + d)
    dx = 1.0 / max(N)
    dt = 0.2 * dx * dx / nu
    return prob, nu, dx, dt


def _run_parts(d, N, P, T, precision):
    prob, nu, dx, dt = _case(d, N)
    th0 = torch.from_numpy(prob.theta(N, dx)).cuda()
    g0 = torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda()
    parts = [lb.Slab(d, N, p, P, nu, dx, dt, precision, theta_ref=1.5) for p in range(P)]
    mx = float(th0.abs().max())
    for s in parts:
        s.set_theta0(SL.with_ghost_layers(th0, s.z0, s.nz), SL.with_ghost_layers(g0, s.z0, s.nz, vector=True), mx)
    send = [s.halo_buffers(2) for s in parts]
    recv = [s.halo_buffers(2) for s in parts]

    def exchange():
        for p, s in enumerate(parts):
            s.pack(send[p][0], send[p][1])
        for p, s in enumerate(parts):
            recv[p][0].copy_(send[(p - 1) % P][1])  # lower ghost <- the part below's "up"
            recv[p][1].copy_(send[(p + 1) % P][0])  # upper ghost <- the part above's "down"
            s.unpack(recv[p][0], recv[p][1])

    for _ in range(T):
        exchange()
        for s in parts:
            s.step()
    exchange()
    fields = [s.macros() for s in parts]
    total = sum(s.sum_theta() for s in parts)
    th = torch.cat([f[0] for f in fields], 0)
    g = torch.cat([f[1] for f in fields], 1)
    u = torch.cat([f[2] for f in fields], 1)
    for s in parts:
        s.close()
    return (th, g, u), total, (prob, nu, dx, dt, th0, g0)


CASES = [(2, (70, 45), 1, 13), (2, (70, 45), 2, 13), (2, (64, 33), 3, 11), (2, (5, 9), 4, 6),
         (3, (20, 13, 9), 2, 7), (3, (16, 8, 6), 3, 5), (4, (10, 8, 6, 5), 2, 4)]


@pytest.mark.parametrize("precision", ["fx64", "fp64", "fp32s"])
@pytest.mark.parametrize("d,N,P,T", CASES)
def test_slabs_equal_the_single_grid_bitwise(d, N, P, T, precision):
    (th, g, u), total, (prob, nu, dx, dt, th0, g0) = _run_parts(d, N, P, T, precision)
    s = lb.Solver(d, N, nu, dx, dt, precision=precision, theta_ref=1.5)
    s.set_theta0(th0, g0)
    s.step(T)
    th1, g1, u1 = s.macros()
    torch.cuda.synchronize()
    assert torch.equal(th, th1) and torch.equal(g, g1) and torch.equal(u, u1)
    assert total == pytest.approx(s.sum_theta(), rel=1e-14)
    s.close()


@pytest.mark.parametrize("d,N,P,T", [(2, (70, 45), 3, 13), (3, (20, 13, 9), 2, 7)])
def test_slabs_match_the_oracle(d, N, P, T):
    (th, g, u), total, (prob, nu, dx, dt, th0, g0) = _run_parts(d, N, P, T, "fx64")
    m = O.Model(d, N, nu, dx, dt)
    f = m.run(m.initialize(prob.theta(N, dx), prob.grad(N, dx)), T)
    ref = m.recover(f)
    for a, b in zip((th, g, u), ref):
        a = a.cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    assert total == pytest.approx(m.total(f), rel=1e-13)


def test_slab_refuses_stale_ghost_layers_and_missing_gradient():
    d, N = 2, (40, 30)
    prob, nu, dx, dt = _case(d, N)
    th0 = torch.from_numpy(prob.theta(N, dx)).cuda()
    g0 = torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda()
    s = lb.Slab(d, N, 0, 2, nu, dx, dt, "fx64")
    th_e, g_e = SL.with_ghost_layers(th0, s.z0, s.nz), SL.with_ghost_layers(g0, s.z0, s.nz, vector=True)
    with pytest.raises(lb.LBError) as ei:
        s.set_theta0(th_e, None, float(th0.max()))
    assert ei.value.status == lb.LB_EINVAL
    with pytest.raises(lb.LBError) as ei:  # this part's max beyond the stated grid maximum
        s.set_theta0(th_e, g_e, 0.5 * float(th0.max()))
    assert ei.value.status == lb.LB_EINVAL
    s.set_theta0(th_e, g_e, float(th0.max()))
    s.step()  # right after the initialisation the ghost layers are current
    with pytest.raises(lb.LBError) as ei:
        s.step()
    assert ei.value.status == lb.LB_ESTATE
    with pytest.raises(lb.LBError) as ei:
        s.macros()
    assert ei.value.status == lb.LB_ESTATE
    with pytest.raises(lb.LBError):
        lb.Slab(d, N, 2, 2, nu, dx, dt)  # part out of range
    s.close()


def test_one_part_runner_wraps_onto_itself():
    """SlabRunner with one part (no process group): its exchange wraps the
    buffers onto the part itself and the result is the single grid's."""
    d, N, T = 2, (48, 20), 9
    prob, nu, dx, dt = _case(d, N)
    th0 = torch.from_numpy(prob.theta(N, dx)).cuda()
    g0 = torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda()
    r = SL.SlabRunner(d, N, nu, dx, dt, "fx64", rank=0, world=1)
    r.set_theta0(th0, g0)
    r.step(T)
    th, _, u = r.macros()
    s = lb.Solver(d, N, nu, dx, dt, precision="fx64")
    s.set_theta0(th0, g0)
    s.step(T)
    th1, _, u1 = s.macros()
    assert torch.equal(th, th1) and torch.equal(u, u1)
    assert r.sum_theta() == pytest.approx(s.sum_theta(), rel=1e-14)
