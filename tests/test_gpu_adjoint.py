"""GPU discrete adjoint: against the FP64 oracle adjoint (the CPU reference
gradient, itself pinned by finite differences), against central finite
differences of the GPU forward on 16 random directions, independent of the
checkpoint interval, and through torch.autograd."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W
from paper_2309_02825_gb300.adjoint import burgers_velocity

pytestmark = pytest.mark.gpu


def _case(d, N, T, seed):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.05, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2048 * dx * dx / nu
    rng = np.random.default_rng(seed + 1)
    tgt = W.FourierProblem(d, nu, prob.offset, prob.k, prob.amp + rng.normal(0, 0.01, len(prob.amp)), prob.phase)
    return prob.theta(N, dx), np.ascontiguousarray(tgt.u(N, dx, T * dt)), nu, dx, dt


def _gpu_grad(d, N, nu, dx, dt, T, th0, ut, precision="fp64", C=0):
    s = lb.Solver(d, N, nu, dx, dt, precision=precision)
    a = lb.Adjoint(s, T, checkpoint=C, want_nu=True)
    u = a.forward(torch.from_numpy(th0).cuda())
    r = u - torch.from_numpy(ut).cuda()
    a.seed(r.contiguous())
    a.step(T)
    g, dnu = a.result()
    L = 0.5 * float((r * r).sum())
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
    assert L == pytest.approx(Lo, rel=1e-9)
    rel = np.max(np.abs(g - go)) / np.max(np.abs(go))
    print("adjoint %s d=%d N=%s T=%d: dtheta0 rel %.2e, dnu rel %.2e" % (precision, d, N, T, rel, abs(dnu / dnuo - 1)))
    assert rel <= 1e-9
    assert dnu == pytest.approx(dnuo, rel=1e-9)


def test_adjoint_checkpoint_interval_does_not_change_the_gradient():
    d, N, T = 2, (70, 45), 23
    th0, ut, nu, dx, dt = _case(d, N, T, 9)
    ref = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, C=1)
    for C in (0, 5, 23):
        L, g, dnu = _gpu_grad(d, N, nu, dx, dt, T, th0, ut, C=C)
        assert np.array_equal(g, ref[1]) and dnu == ref[2]


@pytest.mark.parametrize("precision", ["fp64", "fx64", "fp32s"])
def test_recorded_segments_match_single_steps(precision):
    """Whole checkpoint segments run as recorded graphs (C forward sweeps; C - 1
    recompute sweeps and C reverse steps); one reverse step per call, or calls
    that split segments, launch the same kernels one by one.  The gradient and
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
    assert rel <= 1e-9
