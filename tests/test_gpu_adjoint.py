"""GPU discrete adjoint: against the FP64 oracle adjoint (the CPU reference
gradient, itself pinned by finite differences), against central finite
differences of the GPU forward on 16 random directions, independent of the
checkpoint interval, and through torch.autograd."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W
from paper_2309_02825_gb300.adjoint import burgers_velocity

pytestmark = pytest.mark.gpu

# GPU vs oracle (FP64 and 64-bit fixed-point states): max-norm relative
# difference of dL/dtheta0, and relative difference of L and dL/dnu
TOL = 1e-12


def _case(d, N, T, seed):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.05, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2048 * dx * dx / nu
    rng = np.random.default_rng(seed + 1)
    tgt = W.FourierProblem(d, nu, prob.offset, prob.k, prob.amp + rng.normal(0, 0.01, len(prob.amp)), prob.phase)
    return prob.theta(N, dx), np.ascontiguousarray(tgt.u(N, dx, T * dt)), nu, dx, dt


def _gpu_grad(d, N, nu, dx, dt, T, th0, ut, precision="fp64", C=0, tt=None):
    """L = 1/2 |u(T) - ut|^2 [+ 1/2 |theta(T) - tt|^2] and its gradients."""
    s = lb.Solver(d, N, nu, dx, dt, precision=precision)
    a = lb.Adjoint(s, T, checkpoint=C, want_nu=True)
    th = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    u = a.forward(torch.from_numpy(th0).cuda(), theta=th)
    r = u - torch.from_numpy(ut).cuda()
    L = 0.5 * float((r * r).sum())
    rt = None
    if tt is not None:
        rt = (th - torch.from_numpy(tt).cuda()).contiguous()
        L += 0.5 * float((rt * rt).sum())
    a.seed(r.contiguous(), rt)
    a.step(T)
    g, dnu = a.result()
    a.close()
    s.close()
    return L, g.cpu().numpy(), dnu


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("d,N,T", [(1, (100,), 37), (2, (70, 45), 23), (2, (10, 8), 12), (3, (20, 13, 9), 7)])
def test_adjoint_matches_oracle(d, N, T, precision):
    th0, ut, nu, dx, dt = _case(d, N, T, 40 + d)
    m = O.Model(d, N, nu, dx, dt)
    Lo, go, dnuo = m.adjoint(th0, ut, T)
    L, g, dnu = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, precision)
    rel = np.max(np.abs(g - go)) / np.max(np.abs(go))
    print("adjoint %s d=%d N=%s T=%d: L rel %.2e, dtheta0 rel %.2e, dnu rel %.2e"
          % (precision, d, N, T, abs(L / Lo - 1), rel, abs(dnu / dnuo - 1)))
    assert L == pytest.approx(Lo, rel=TOL)
    assert rel <= TOL
    assert dnu == pytest.approx(dnuo, rel=TOL)


def test_adjoint_checkpoint_interval_does_not_change_the_gradient():
    d, N, T = 2, (70, 45), 23
    th0, ut, nu, dx, dt = _case(d, N, T, 9)
    ref = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, C=1)
    for C in (0, 5, 23):
        L, g, dnu = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, C=C)
        assert np.array_equal(g, ref[1]) and dnu == ref[2]


@pytest.mark.parametrize("precision", ["fp64", "fx64", "fp32s"])
def test_recorded_segments_match_single_steps(precision):
    """Whole checkpoint segments run as recorded graphs (C forward sweeps; C
    reverse steps with the previous segment's C - 1 recompute sweeps on a
    second branch); one reverse step per call, or calls that split segments,
    recompute and reverse one segment at a time with single launches.  The gradient and
    dL/dnu agree bit for bit, also on a second forward and seed of the same
    workspace (graphs reused or re-recorded)."""
    d, N, T = 2, (70, 45), 23  # C = 5: four whole segments and a short last one
    th0, ut, nu, dx, dt = _case(d, N, T, 21)
    s = lb.Solver(d, N, nu, dx, dt, precision=precision)
    a = lb.Adjoint(s, T, want_nu=True)

    def run(steps):
        u = a.forward(torch.from_numpy(th0).cuda())
        a.seed((u - torch.from_numpy(ut).cuda()).contiguous())
        for n in steps:
            a.step(n)
        g, dnu = a.result()
        return g.cpu().numpy(), dnu

    ref = run([T])
    for steps in ([1] * T, [7, 16], [T]):
        g, dnu = run(steps)
        assert np.array_equal(g, ref[0]) and dnu == ref[1], steps
    a.close()
    s.close()


def test_adjoint_matches_gpu_finite_differences():
    d, N, T = 2, (128, 128), 200
    th0, ut, nu, dx, dt = _case(d, N, T, 17)
    L, g, dnu = _gpu_grad(d, N, nu, dx, dt, T, th0, ut)

    def loss(th, nu_):
        s = lb.Solver(d, N, nu_, dx, dt)
        a = lb.Adjoint(s, T, want_nu=False)
        u = a.forward(torch.from_numpy(np.ascontiguousarray(th)).cuda())
        r = u - torch.from_numpy(ut).cuda()
        v = 0.5 * float((r * r).sum())
        a.close()
        s.close()
        return v

    rng = np.random.default_rng(3)
    for _ in range(16):
        v = rng.normal(size=th0.shape)
        h = 1e-5
        fd = (loss(th0 + h * v, nu) - loss(th0 - h * v, nu)) / (2 * h)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)
    hn = 1e-6 * nu
    fd = (loss(th0, nu + hn) - loss(th0, nu - hn)) / (2 * hn)
    assert dnu == pytest.approx(fd, rel=1e-6)


def test_autograd_function():
    d, N, T = 2, (64, 48), 30
    th0, ut, nu, dx, dt = _case(d, N, T, 5)
    theta0 = torch.from_numpy(th0).cuda().requires_grad_(True)
    nu_t = torch.tensor(nu, dtype=torch.float64, device="cuda", requires_grad=True)
    u = burgers_velocity(theta0, nu_t, d, N, dx, dt, T)
    loss = 0.5 * ((u - torch.from_numpy(ut).cuda()) ** 2).sum()
    loss.backward()
    L, g, dnu = _gpu_grad(d, N, nu, dx, dt, T, th0, ut)
    assert float(loss.detach()) == pytest.approx(L, rel=1e-14)
    assert np.array_equal(theta0.grad.cpu().numpy(), g)
    assert float(nu_t.grad) == dnu


@pytest.mark.parametrize("d,N,T", [(1, (100,), 37), (2, (70, 45), 23), (3, (20, 13, 9), 7)])
def test_fp32_shifted_adjoint_tracks_fp64(d, N, T):
    """FP32 shifted storage: the forward states carry float rounding and the
    reverse pass computes in FP32, so the gradient differs from the FP64 one
    by float rounding relative to the velocity misfit (~1e-5 here)."""
    th0, ut, nu, dx, dt = _case(d, N, T, 60 + d)
    L64, g64, dnu64 = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, "fp64")
    L32, g32, dnu32 = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, "fp32s")
    rel = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    print("fp32s adjoint d=%d: dtheta0 rel %.2e, dnu rel %.2e, L rel %.2e" % (d, rel, abs(dnu32 / dnu64 - 1), abs(L32 / L64 - 1)))
    assert rel <= 1e-3
    assert dnu32 == pytest.approx(dnu64, rel=1e-3)


@pytest.mark.parametrize("d,N,T", [(1, (100,), 37), (2, (70, 45), 23), (3, (20, 13, 9), 7)])
def test_fx64_theta0_gradient_without_nu(d, N, T):
    """Fixed-point states, dL/dtheta0 only: the reverse pass is then entirely
    integer (K^T on round(phi 2^G)); it must meet the same bar against the
    oracle as the FP64 adjoint."""
    th0, ut, nu, dx, dt = _case(d, N, T, 70 + d)
    m = O.Model(d, N, nu, dx, dt)
    _, go, _ = m.adjoint(th0, ut, T)
    s = lb.Solver(d, N, nu, dx, dt, precision="fx64")
    a = lb.Adjoint(s, T, want_nu=False)
    u = a.forward(torch.from_numpy(th0).cuda())
    a.seed((u - torch.from_numpy(ut).cuda()).contiguous())
    a.step(T)
    g, _ = a.result()
    g = g.cpu().numpy()
    rel = np.max(np.abs(g - go)) / np.max(np.abs(go))
    print("fx64 theta0-only adjoint d=%d: rel %.2e" % (d, rel))
    assert rel <= TOL


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("d,N,T", [(1, (100,), 37), (2, (70, 45), 23), (3, (20, 13, 9), 7)])
def test_theta_seed_matches_oracle(d, N, T, precision):
    """A loss on theta(T) as well as u(T): lb_adjoint_seed's dL/dtheta term
    against the oracle adjoint of L = 1/2|u - ut|^2 + 1/2|theta - tt|^2."""
    th0, ut, nu, dx, dt = _case(d, N, T, 80 + d)
    tt = th0 * (1.0 + 0.01 * np.sin(np.arange(th0.size)).reshape(th0.shape))
    m = O.Model(d, N, nu, dx, dt)
    Lo, go, dnuo = m.adjoint(th0, ut, T, theta_target=tt)
    L, g, dnu = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, precision, tt=tt)
    rel = np.max(np.abs(g - go)) / np.max(np.abs(go))
    print("theta-seed adjoint %s d=%d: L rel %.2e, dtheta0 rel %.2e, dnu rel %.2e"
          % (precision, d, abs(L / Lo - 1), rel, abs(dnu / dnuo - 1)))
    assert L == pytest.approx(Lo, rel=TOL)
    assert rel <= TOL
    assert dnu == pytest.approx(dnuo, rel=TOL)


def test_theta_only_seed_and_empty_seed():
    """dL/du may be omitted (a loss of theta alone); omitting both is
    LB_EINVAL.  The oracle's reference is its adjoint with the u target set
    to its own u(T), so that only the theta term contributes."""
    d, N, T = 2, (40, 30), 9
    th0, _, nu, dx, dt = _case(d, N, T, 88)
    tt = th0 * 1.002
    m = O.Model(d, N, nu, dx, dt)
    _, _, u_own = m.recover(m.run(m.initialize(th0), T))
    _, go, dnuo = m.adjoint(th0, u_own, T, theta_target=tt)
    s = lb.Solver(d, N, nu, dx, dt)
    a = lb.Adjoint(s, T, want_nu=True)
    th = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    a.forward(torch.from_numpy(th0).cuda(), theta=th)
    with pytest.raises(lb.LBError) as ei:
        a.seed(None, None)
    assert ei.value.status == lb.LB_EINVAL
    a.seed(None, (th - torch.from_numpy(tt).cuda()).contiguous())
    a.step(T)
    g, dnu = a.result()
    assert np.max(np.abs(g.cpu().numpy() - go)) <= TOL * np.max(np.abs(go))
    assert dnu == pytest.approx(dnuo, rel=TOL)
    a.close()
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_adjoint_at_512_squared_2000_steps_matches_oracle(precision):
    """The adjoint workload at full size: 512^2 D2Q9, nu = 0.02, eps = 0.2048,
    T = 2000, theta0 = 1.5 + 6 seeded modes, target from perturbed amplitudes.
    The oracle gradient comes from its checkpointed adjoint (every 45th state
    kept, segments recomputed; bit-identical to keeping all states) run on
    every host core."""
    case = W.adjoint_2d(512, 2000)
    N, d, T = case.N, case.d, case.nsteps
    th0 = case.problem.theta(N, case.dx)
    ut = np.ascontiguousarray(case.extra["target"].u(N, case.dx, T * case.dt))
    O.set_threads(os.cpu_count() or 1)
    m = O.Model(d, N, case.nu, case.dx, case.dt)
    Lo, go, dnuo = m.adjoint(th0, ut, T, checkpoint=45)
    L, g, dnu = _gpu_grad(d, N, case.nu, case.dx, case.dt, T, th0, ut, precision)
    rel = np.max(np.abs(g - go)) / np.max(np.abs(go))
    print("adjoint 512^2 T=2000 %s: L rel %.2e, dtheta0 rel %.2e, dnu rel %.2e"
          % (precision, abs(L / Lo - 1), rel, abs(dnu / dnuo - 1)))
    assert L == pytest.approx(Lo, rel=TOL)
    assert rel <= TOL
    assert dnu == pytest.approx(dnuo, rel=TOL)


def test_autograd_reuses_its_workspace_and_supports_retain_graph():
    """Ten iterations of a training loop on theta0 and nu create one solver
    and workspace; the viscosity is changed in place.  Two backward passes of
    one graph (retain_graph) give identical gradients, also after another
    forward has run in the same workspace in between."""
    from paper_2309_02825_gb300 import adjoint as A
    A.clear_cache()
    d, N, T = 2, (64, 48), 30
    th0, ut, nu, dx, dt = _case(d, N, T, 5)
    ut_t = torch.from_numpy(ut).cuda()
    theta0 = torch.from_numpy(th0).cuda().requires_grad_(True)
    nu_t = torch.tensor(nu, dtype=torch.float64, device="cuda", requires_grad=True)
    created = A.stats["workspaces_created"]
    free0 = None
    for it in range(10):
        u = burgers_velocity(theta0, nu_t, d, N, dx, dt, T)
        loss = 0.5 * ((u - ut_t) ** 2).sum()
        loss.backward()
        with torch.no_grad():
            theta0 -= 1e-3 * theta0.grad
            nu_t -= 1e-4 * nu * torch.sign(nu_t.grad)
        theta0.grad = None
        nu_t.grad = None
        torch.cuda.synchronize()
        if it == 0:
            free0 = torch.cuda.mem_get_info()[0]
    assert A.stats["workspaces_created"] == created + 1
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    # retain_graph: the second backward replays the same reverse pass
    u = burgers_velocity(theta0, nu_t, d, N, dx, dt, T)
    loss = 0.5 * ((u - ut_t) ** 2).sum()
    g1 = torch.autograd.grad(loss, [theta0, nu_t], retain_graph=True)
    other = burgers_velocity(theta0.detach() * 1.01, nu_t, d, N, dx, dt, T)  # same workspace: overwrites the states
    replays = A.stats["forward_replays"]
    g2 = torch.autograd.grad(loss, [theta0, nu_t])
    assert A.stats["forward_replays"] == replays + 1
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])
    del other
    # against a fresh solver at the final parameters
    L, g, dnu = _gpu_grad(d, N, float(nu_t.detach()), dx, dt, T, theta0.detach().cpu().numpy(), ut)
    assert np.array_equal(g1[0].cpu().numpy(), g) and float(g1[1]) == dnu


def test_autograd_theta_output_matches_oracle():
    from paper_2309_02825_gb300.adjoint import burgers_fields
    d, N, T = 2, (40, 30), 11
    th0, ut, nu, dx, dt = _case(d, N, T, 91)
    tt = th0 * 0.999
    theta0 = torch.from_numpy(th0).cuda().requires_grad_(True)
    nu_t = torch.tensor(nu, dtype=torch.float64, device="cuda", requires_grad=True)
    u, th = burgers_fields(theta0, nu_t, d, N, dx, dt, T)
    loss = 0.5 * ((u - torch.from_numpy(ut).cuda()) ** 2).sum() + 0.5 * ((th - torch.from_numpy(tt).cuda()) ** 2).sum()
    loss.backward()
    Lo, go, dnuo = O.Model(d, N, nu, dx, dt).adjoint(th0, ut, T, theta_target=tt)
    assert float(loss.detach()) == pytest.approx(Lo, rel=TOL)
    g = theta0.grad.cpu().numpy()
    assert np.max(np.abs(g - go)) <= TOL * np.max(np.abs(go))
    assert float(nu_t.grad) == pytest.approx(dnuo, rel=TOL)
