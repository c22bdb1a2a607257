"""Batched 2D instances: bit-identical to the single-instance solver under
every schedule (same kernel arithmetic), and within the FP64 / FP32 bounds
of the oracle per instance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = [(70, 45), (5, 7), (33, 20), (130, 3), (64, 64), (1, 9), (200, 17)]
NUS = [0.02, 0.005, 0.08, 0.03, 0.011, 0.05, 0.1]


def _setup(seed=7):
    probs, dxs, dts, th0, g0 = [], [], [], [], []
    for j, ((n0, n1), nu) in enumerate(zip(SIZES, NUS)):
        p = W.FourierProblem.random(2, nu, 6, 3, 0.05, 1.5, seed + j)
        dx = 1.0 / max(n0, n1)
        dt = 4.0 * dx * dx
        probs.append(p)
        dxs.append(dx)
        dts.append(dt)
        th0.append(p.theta((n0, n1), dx).ravel())
        g0.append(np.ascontiguousarray(p.grad((n0, n1), dx)).ravel())
    return probs, dxs, dts, np.concatenate(th0), np.concatenate(g0)


def _single(j, prob, dx, dt, n, precision, theta_ref):
    N = SIZES[j]
    s = lb.Solver(2, N, prob.nu, dx, dt, precision=precision, theta_ref=theta_ref)
    s.set_theta0(torch.from_numpy(prob.theta(N, dx)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda())
    s.step(n)
    th, _, u = s.macros()
    return th, u


@pytest.mark.parametrize("precision", ["fp32s", "fp64", "fx64"])
@pytest.mark.parametrize("sched", [(96e6, 256, True), (0.0, 128, False), (40e3, 512, True), (1e18, 256, True),
                                   (1e18, 64, True)])
def test_batch_equals_single_instance_bitwise(precision, sched):
    probs, dxs, dts, th0, g0 = _setup()
    n = 37  # one recorded 32-step graph plus 5 direct launches, odd parity
    b = lb.Batch(SIZES, NUS, dxs, dts, precision=precision, theta_ref=[1.5] * len(SIZES))
    b.set_schedule(*sched)
    b.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    b.step(n)
    th, u = b.macros()
    ths, us = b.split(th), b.split(u, 2)
    for j in range(len(SIZES)):
        t1, u1 = _single(j, probs[j], dxs[j], dts[j], n, precision, 1.5)
        assert torch.equal(ths[j], t1), j
        assert torch.equal(us[j], u1), j


# blocked launches (steps per launch, tile edge, threads): tiles wider and
# narrower than the instances, tiles that do not divide them, a remainder
# launch (37 = 9 x 4 + 1, 12 x 3 + 1, 4 x 8 + 5), graphs of 16 launches
# (1 step per launch)
BLOCKED = [(4, 28, 512), (3, 17, 256), (8, 22, 1024), (1, 33, 256), (2, 5, 512)]


@pytest.mark.parametrize("precision,blk", [(p, b) for p in ("fp32s", "fp64", "fx64") for b in BLOCKED]
                         + [("fp32s", (4, 48, 1024)), ("fp32s", (6, 40, 512))])
def test_blocked_batch_equals_single_instance_bitwise(precision, blk):
    """K steps per launch in shared memory: every instance still evolves bit
    for bit as the single-grid solver does, across remainder launches, graph
    replays and a switch back to one launch per step."""
    probs, dxs, dts, th0, g0 = _setup()
    b = lb.Batch(SIZES, NUS, dxs, dts, precision=precision, theta_ref=[1.5] * len(SIZES))
    b.set_blocking(*blk)
    sch = b.schedule()
    assert sch["steps_per_launch"] == blk[0] and sch["tile"] == blk[1] and sch["tiles"] > 0
    b.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    b.step(37)
    b.set_schedule(96e6, 128, True)
    b.step(3)
    b.set_blocking(*blk)
    b.step(20)
    n = 60
    th, u = b.macros()
    ths, us = b.split(th), b.split(u, 2)
    for j in range(len(SIZES)):
        t1, u1 = _single(j, probs[j], dxs[j], dts[j], n, precision, 1.5)
        assert torch.equal(ths[j], t1), j
        assert torch.equal(us[j], u1), j


def test_blocked_rejects_tiles_beyond_shared_memory():
    probs, dxs, dts, th0, g0 = _setup()
    b = lb.Batch(SIZES, NUS, dxs, dts, precision="fx64")
    with pytest.raises(lb.LBError) as ei:
        b.set_blocking(8, 200, 512)
    assert ei.value.status == lb.LB_EINVAL
    with pytest.raises(lb.LBError) as ei:
        b.set_blocking(4, 20, 300)
    assert ei.value.status == lb.LB_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_batch_fp64_matches_oracle(precision):
    probs, dxs, dts, th0, g0 = _setup(11)
    n = 20
    b = lb.Batch(SIZES, NUS, dxs, dts, precision=precision)
    b.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    b.step(n)
    th, u = b.macros()
    ths, us = b.split(th), b.split(u, 2)
    for j, N in enumerate(SIZES):
        m = O.Model(2, N, NUS[j], dxs[j], dts[j])
        p = probs[j]
        tho, _, uo = m.recover(m.run(m.initialize(p.theta(N, dxs[j]), p.grad(N, dxs[j])), n))
        assert np.max(np.abs(ths[j].cpu().numpy() - tho)) <= 1e-12 * np.max(np.abs(tho))
        assert np.max(np.abs(us[j].cpu().numpy() - uo)) <= 1e-12 * np.max(np.abs(uo))


def test_batch_autotune_and_errors():
    probs, dxs, dts, th0, g0 = _setup(3)
    b = lb.Batch(SIZES, NUS, dxs, dts, precision="fp32s", theta_ref=[1.5] * len(SIZES))
    choice = b.autotune(4)
    assert choice["threads"] in (64, 128, 256, 512, 1024) and choice["groups"] >= 1 and choice["us_per_step"] > 0
    assert choice["steps_per_launch"] in (0, 2, 3, 4, 5, 6, 8, 12)
    b.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    n = 40
    b.step(n)
    th, u = b.macros()
    ex_t = np.concatenate([p.theta(N, dxs[j], n * dts[j]).ravel() for j, (p, N) in enumerate(zip(probs, SIZES))])
    ex_u = np.concatenate([np.ascontiguousarray(p.u(N, dxs[j], n * dts[j])).ravel()
                           for j, (p, N) in enumerate(zip(probs, SIZES))])
    err = b.errors(th, u, torch.from_numpy(ex_t).cuda(), torch.from_numpy(ex_u).cuda())
    tht, ut = th.cpu().numpy(), u.cpu().numpy()
    for j, N in enumerate(SIZES):
        a, z = b.node_off[j], b.node_off[j + 1]
        et = tht[a:z] - ex_t[a:z]
        eu = (ut[2 * a:2 * z] - ex_u[2 * a:2 * z]).reshape(2, -1)
        assert err[j, 0] == pytest.approx(np.sqrt(np.mean(et ** 2)), rel=1e-12)
        assert err[j, 1] == pytest.approx(np.sqrt(np.mean(np.sum(eu ** 2, axis=0))), rel=1e-12)
        assert err[j, 2] == pytest.approx(np.max(np.abs(et)), rel=1e-15)
