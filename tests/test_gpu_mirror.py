"""GPU parity on grids with mirror walls (zero normal velocity; the paper's
Example 1) against the oracle's wall model: the periodic FP64 oracle on the
grid doubled by even reflection, restricted to the original nodes.

The CUDA path folds the doubled grid back (reflected rows and populations in
the pull, x-reflected halo scalars at the wall nodes), so agreement here
checks that folding node by node.  Grids span several warp segments with
ragged tails, every lattice (D1Q3 .. D4Q33), mixed periodic/mirror axes and
the smallest mirror axis (3 nodes).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    return t.detach().cpu().numpy()


def _kinds(mirror):
    return ["mirror" if m else "periodic" for m in mirror]


def _run_both(d, N, mirror, nsteps, precision="fp64", grad=True, seed=17, theta_ref=1.5):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.1, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2 * dx * dx / nu
    th0 = prob.theta(N, dx)
    g0 = prob.grad(N, dx) if grad else None
    m = O.MirrorModel(d, N, mirror, nu, dx, dt)
    ref = m.recover(m.run(m.initialize(th0, g0), nsteps))
    s = lb.Solver(d, N, nu, dx, dt, precision=precision, theta_ref=theta_ref, boundary=_kinds(mirror))
    s.set_theta0(_dev(th0), None if g0 is None else _dev(g0))
    s.step(nsteps)
    got = [_host(t) for t in s.macros()]
    torch.cuda.synchronize()
    return ref, got, s, m, th0


def _bounds(ref, m, nsteps, eps_rel, scale_theta, growth):
    """Absolute bounds per field: rounding floor of J = sum e f (terms of
    size scale_theta), carried over nsteps (growth(n)), times the recovery
    coefficient of each field."""
    p = m.params
    sigma = 2 * p["w1"] + 4 * (m.full.d - 1) * p["wd"]
    floor_j = 8 * m.q * eps_rel * scale_theta * growth(nsteps + 1)
    return {"theta": floor_j, "grad": floor_j * p["s1"] / (sigma * p["dx"]),
            "u": floor_j * (2 - p["s1"]) * p["c"] / np.min(ref[0])}


def _check(ref, got, m, nsteps, precision, th0):
    if precision == "fp32s":
        # FP32 shifted storage: every stored value rounds once per step (the
        # FP32 test's bound, linear in the step count)
        A = float(np.max(np.abs(th0 - 1.5)))
        tol = _bounds(ref, m, nsteps, EPS32, A, float)
    else:
        b = _bounds(ref, m, nsteps, EPS64, np.max(np.abs(ref[0])), np.sqrt)
        tol = {k: TOL64 * float(np.max(np.abs(r))) + (b[k] if k != "theta" else 0.0)
               for k, r in zip(("theta", "grad", "u"), ref)}
    rel = {}
    for name, a, r in zip(("theta", "grad", "u"), got, ref):
        diff = float(np.max(np.abs(a - r)))
        rel[name] = diff / max(float(np.max(np.abs(r))), 1e-300)
        assert diff <= tol[name], (name, diff, tol[name])
    return rel


CASES = [
    (1, (100,), (1,), 1), (1, (100,), (1,), 37), (1, (3,), (1,), 9), (1, (65,), (1,), 20), (1, (129,), (1,), 13),
    (2, (70, 45), (1, 1), 23), (2, (70, 45), (1, 0), 11), (2, (70, 45), (0, 1), 11), (2, (3, 33), (1, 1), 6),
    (2, (130, 3), (0, 1), 7), (2, (64, 64), (1, 1), 20), (2, (200, 17), (1, 1), 60),
    (3, (37, 22, 13), (1, 1, 1), 9), (3, (37, 22, 13), (0, 1, 0), 5), (3, (3, 4, 5), (1, 1, 1), 5),
    (3, (64, 16, 8), (1, 0, 1), 8),
    (4, (10, 8, 6, 5), (1, 1, 1, 1), 6), (4, (10, 8, 6, 5), (0, 0, 1, 1), 4), (4, (3, 4, 3, 5), (1, 0, 1, 0), 3),
]


@pytest.mark.parametrize("precision", ["fp64", "fx64", "fp32s"])
@pytest.mark.parametrize("d,N,mirror,nsteps", CASES)
def test_mirror_matches_oracle(d, N, mirror, nsteps, precision):
    ref, got, _, m, th0 = _run_both(d, N, mirror, nsteps, precision)
    rel = _check(ref, got, m, nsteps, precision, th0)
    print("mirror %s d=%d N=%s walls=%s steps=%d rel %s" % (precision, d, N, mirror, nsteps, rel))


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("d,N,mirror", [(1, (50,), (1,)), (2, (66, 40), (1, 1)), (3, (20, 18, 9), (1, 0, 1))])
def test_mirror_fd_gradient_fallback(d, N, mirror, precision):
    ref, got, _, m, th0 = _run_both(d, N, mirror, 5, precision, grad=False)
    _check(ref, got, m, 5, precision, th0)


def test_mirror_graph_replay_matches_single_steps():
    """lb_step(70) replays recorded 32-sweep graphs; the same state results
    from 70 calls of one step (fixed point: bit for bit)."""
    _, _, s, _, th0 = _run_both(2, (70, 45), (1, 1), 0, "fx64")
    s2 = lb.Solver(2, (70, 45), s.params["nu"], s.params["dx"], s.params["dt"], precision="fx64",
                   boundary=["mirror", "mirror"])
    prob = W.FourierProblem.random(2, 0.02, 6, 3, 0.1, 1.5, 17)
    g0 = _dev(prob.grad((70, 45), s.params["dx"]))
    s.set_theta0(_dev(th0), g0)
    s2.set_theta0(_dev(th0), g0)
    s.step(70)
    for _ in range(70):
        s2.step(1)
    assert torch.equal(s.save_state(), s2.save_state())


@pytest.mark.parametrize("d,N,mirror", [(1, (77,), (1,)), (2, (70, 45), (1, 0)), (3, (24, 10, 7), (1, 1, 1))])
def test_mirror_fx64_wall_weighted_total_exact(d, N, mirror):
    """Fixed point: the total weighted by 1/2 per wall a node lies on is an
    exact invariant; in integers, with weights 2^(k - walls), it never
    changes, and lb_sum_theta equals the oracle's doubled total / 2^k."""
    ref, got, s, m, th0 = _run_both(d, N, mirror, 0, "fx64")
    pitch, slab, _ = s.state_layout()
    q = int(s.params["q"])
    k = sum(mirror)
    w = torch.from_numpy((m.wall_weights() * 2 ** k).astype(np.int64)).cuda()

    def itotal():
        st = s.save_state().view(torch.int64).view(q, *reversed(N[1:]), pitch)[..., : N[0]]
        return int((st * w[None]).sum().item())

    t0, h0 = itotal(), s.sum_theta()
    assert abs(h0 - float(np.sum(m.wall_weights() * th0))) <= 1e-14 * abs(h0)
    s.step(41)
    assert itotal() == t0
    assert abs(s.sum_theta() - h0) <= 1e-14 * abs(h0)


@pytest.mark.parametrize("precision", ["fp64", "fp32s"])
def test_mirror_weighted_total_matches_oracle(precision):
    d, N, mirror, n = 2, (70, 45), (0, 1), 30
    ref, got, s, m, th0 = _run_both(d, N, mirror, n, precision)
    f = m.run(m.initialize(th0, W.FourierProblem.random(d, 0.02, 6, 3, 0.1, 1.5, 17).grad(N, 1.0 / 70)), n)
    ref_total = m.total(f)
    if precision == "fp64":
        tol = 1e-13 * abs(ref_total)
    else:  # each stored value rounds once per step
        tol = np.prod(N) * m.q * EPS32 * float(np.max(np.abs(th0 - 1.5))) * (n + 1)
    assert abs(s.sum_theta() - ref_total) <= tol


def test_mirror_wall_normal_velocity_vanishes():
    """J . n = 0 on wall nodes: exactly in fixed point (the two pulled
    populations are the same stored value), to rounding in FP64."""
    for precision in ("fx64", "fp64"):
        _, got, _, _, _ = _run_both(2, (70, 45), (1, 1), 17, precision)
        u = got[2]
        walls_x = np.abs(u[0][:, [0, -1]]).max()
        walls_y = np.abs(u[1][[0, -1], :]).max()
        if precision == "fx64":
            assert walls_x == 0.0 and walls_y == 0.0
        else:
            assert max(walls_x, walls_y) <= 1e-13 * np.abs(u).max()


@pytest.mark.parametrize("precision", ["fx64", "fp64"])
@pytest.mark.parametrize("eps", [0.5, 2.0])
def test_example1_on_gpu(eps, precision):
    """The paper's Example 1 through the CUDA path: RMSEs equal the oracle's
    wall model and fall at fourth order (levels 0..3: up to 321 nodes,
    12 800 steps)."""
    errs = {"theta": [], "u": []}
    for level in range(4):
        case = W.wall_example1(eps, level)
        p = case.problem
        s = lb.Solver(1, case.N, case.nu, case.dx, case.dt, precision=precision, boundary=["mirror"])
        s.set_theta0(_dev(p.theta(case.N, case.dx)), _dev(p.grad(case.N, case.dx)))
        s.step(case.nsteps)
        th, _, u = [_host(t) for t in s.macros()]
        T = case.t_end
        e_th = O.rmse(th, p.theta(case.N, case.dx, T))
        e_u = O.rmse(u[0], p.u(case.N, case.dx, T)[0])
        if level <= 1:
            m = O.MirrorModel(1, case.N, (True,), case.nu, case.dx, case.dt)
            th_o, _, u_o = m.recover(m.run(m.initialize(p.theta(case.N, case.dx), p.grad(case.N, case.dx)),
                                           case.nsteps))
            assert abs(e_th - O.rmse(th_o, p.theta(case.N, case.dx, T))) <= 1e-6 * e_th
            assert abs(e_u - O.rmse(u_o[0], p.u(case.N, case.dx, T)[0])) <= 1e-6 * e_u
        errs["theta"].append(e_th)
        errs["u"].append(e_u)
    for var, e in errs.items():
        rates = [math.log2(e[i] / e[i + 1]) for i in range(3)]
        assert abs(rates[-1] - 4.0) <= 0.1, (var, rates)


def test_set_boundary_errors():
    s = lb.Solver(2, (40, 30), 0.02, 0.025, 0.005)
    with pytest.raises(lb.LBError) as ei:
        lb.lb_set_boundary(s.ctx, [2, 0])
    assert ei.value.status == lb.LB_EINVAL
    t = lb.Solver(2, (40, 2), 0.02, 0.025, 0.005)
    with pytest.raises(lb.LBError) as ei:
        lb.lb_set_boundary(t.ctx, ["periodic", "mirror"])
    assert ei.value.status == lb.LB_EINVAL
    th0 = _dev(np.full((30, 40), 1.5))
    s.set_theta0(th0)
    lb.lb_set_boundary(s.ctx, ["mirror", "periodic"])
    assert lb.lb_get_boundary(s.ctx, 2) == ["mirror", "periodic"]
    with pytest.raises(lb.LBError) as ei:
        s.step(1)
    assert ei.value.status == lb.LB_ESTATE
    s.set_theta0(th0)
    s.step(3)
    th, _, u = s.macros()
    assert torch.allclose(th, th0, rtol=0, atol=1e-14) and float(u.abs().max()) <= 1e-14
