"""GPU parity of the FP32 shifted-storage path against the FP64 oracle.

The stored value is f - w theta_ref in float and the collision runs in float
with float-rounded constants, so the scheme differs from the FP64 one by
O(2^-24) per operation and per parameter.  With A = max |theta0 - theta_ref|
(the scale of the stored values) the bound used here is
  |theta_gpu - theta_oracle| <= 8 q 2^-24 A (n + 1)
and the same bound on J = sum e f scaled by the recovery coefficient for
grad theta and u; the recovery itself is FP64 on the GPU.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _run(d, N, nsteps, seed=21, theta_ref=1.5):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.1, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2 * dx * dx / nu
    th0, g0 = prob.theta(N, dx), prob.grad(N, dx)
    m = O.Model(d, N, nu, dx, dt)
    ref = m.recover(m.run(m.initialize(th0, g0), nsteps))
    s = lb.Solver(d, N, nu, dx, dt, precision="fp32s", theta_ref=theta_ref)
    s.set_theta0(_dev(th0), _dev(g0))
    s.step(nsteps)
    got = [t.cpu().numpy() for t in s.macros()]
    A = float(np.max(np.abs(th0 - theta_ref)))
    return ref, got, m, A, s, th0


CASES = [(1, (200,), 1), (1, (200,), 40), (2, (150, 70), 1), (2, (150, 70), 25), (2, (64, 64), 20),
         (2, (3, 130), 6), (3, (140, 20, 9), 1), (3, (140, 20, 9), 12), (3, (5, 4, 3), 5),
         (4, (12, 7, 5, 4), 5),
         # 4D rows with padding, of odd length, and filling whole warps
         (4, (50, 3, 4, 3), 3), (4, (11, 5, 4, 3), 4), (4, (64, 3, 3, 3), 3)]


@pytest.mark.parametrize("d,N,nsteps", CASES)
def test_fp32_shifted_matches_oracle(d, N, nsteps):
    ref, got, m, A, _, _ = _run(d, N, nsteps)
    p = m.params
    sigma = 2 * p["w1"] + 4 * (d - 1) * p["wd"]
    bJ = 8 * m.q * EPS32 * A * (nsteps + 1)
    bounds = {"theta": bJ, "grad": bJ * p["s1"] / (sigma * p["dx"]),
              "u": bJ * (2 - p["s1"]) * p["c"] / np.min(ref[0])}
    msg = []
    for name, a, b in zip(("theta", "grad", "u"), got, ref):
        diff = float(np.max(np.abs(a - b)))
        msg.append("%s %.2e (bound %.2e)" % (name, diff, bounds[name]))
        assert diff <= bounds[name], msg
    print("fp32s d=%d N=%s n=%d: %s" % (d, N, nsteps, "; ".join(msg)))


def test_fp32_shifted_conserves_sum():
    d, N, n = 2, (150, 70), 30
    _, _, m, A, s, th0 = _run(d, N, n)
    total = s.sum_theta()
    nodes = np.prod(N)
    # each stored value rounds once per step; the sum of roundings is bounded
    assert abs(total - th0.sum()) <= nodes * m.q * EPS32 * A * (n + 1)


def test_fp32_shifted_tracks_exact_solution():
    """On the 2D sine family at N = 64 the FP32 shifted error against the
    exact solution stays within a few times the FP64 discretisation error."""
    case = W.sine_2d(64)
    s64 = lb.Solver(2, case.N, case.nu, case.dx, case.dt)
    s32 = lb.Solver(2, case.N, case.nu, case.dx, case.dt, precision="fp32s", theta_ref=2.0)
    th0 = _dev(case.problem.theta(case.N, case.dx))
    g0 = _dev(case.problem.grad(case.N, case.dx))
    T = case.t_end
    et = _dev(case.problem.theta(case.N, case.dx, T))
    eu = _dev(case.problem.u(case.N, case.dx, T))
    errs = []
    for s in (s64, s32):
        s.set_theta0(th0, g0)
        s.step(case.nsteps)
        th, _, u = s.macros()
        errs.append(s.reduce(th, u, et, eu))
    assert errs[1]["u0"]["rmse"] < 3 * errs[0]["u0"]["rmse"]
    assert errs[1]["theta"]["rmse"] < 10 * errs[0]["theta"]["rmse"]


@pytest.mark.parametrize("d,N", [(1, (37,)), (2, (20, 12)), (3, (9, 7, 5))])
def test_fp32s_recovery_sums_match_exact_arithmetic(d, N):
    """The FP32-shifted recovery sums the q stored floats of a node on the
    integer pipes, aligned to the node's largest exponent.  On a loaded state
    whose values span 12 decades, with zeros, subnormals and both signs,
    theta = theta_ref + sum_i P_i(x - e_i), J_a = sum_i e_ia P_i(x - e_i) and
    u = (2 - s1) c J / theta must equal exact arithmetic (math.fsum) to a few
    units of the last place."""
    import math

    dx = 1.0 / max(N)
    s = lb.Solver(d, N, 0.02, dx, 0.2 * dx * dx / 0.02, precision="fp32s", theta_ref=2.0)
    pitch, slab, _ = s.state_layout()
    e = O.lattice(d)
    q = e.shape[0]
    shape = tuple(reversed(N))
    rng = np.random.default_rng(7 + d)
    vals = rng.standard_normal((q,) + shape) * 10.0 ** rng.integers(-12, 0, (q,) + shape)
    r = rng.random(vals.shape)
    vals[r < 0.1] = 0.0
    vals[(r >= 0.1) & (r < 0.15)] = 3e-40 * np.sign(rng.standard_normal(np.count_nonzero((r >= 0.1) & (r < 0.15))))
    vals = vals.astype(np.float32)
    state = np.zeros(q * slab, dtype=np.float32)
    rows = int(np.prod(shape[:-1]))
    for i in range(q):
        plane = state[i * slab:(i + 1) * slab].reshape(rows, pitch)
        plane[:, :N[0]] = vals[i].reshape(rows, N[0])
    s.load_state(torch.from_numpy(state).cuda(), 0)
    th, g, u = [t.cpu().numpy() for t in s.macros()]
    p = s.params
    ucoef = (2.0 - p["s1"]) * p["c"]
    # the pulled values P_i(x - e_i): roll population i by +e_i along each axis (x is the last array axis)
    pulled = [np.roll(vals[i].astype(np.float64), tuple(int(e[i, a]) for a in range(d)),
                      tuple(d - 1 - a for a in range(d))) for i in range(q)]
    th_x = np.empty(shape)
    J_x = np.empty((d,) + shape)
    for idx in np.ndindex(*shape):
        col = [pv[idx] for pv in pulled]
        th_x[idx] = math.fsum([2.0] + col)
        for a in range(d):
            J_x[(a,) + idx] = math.fsum([float(e[i, a]) * col[i] for i in range(q)])
    u_x = ucoef * J_x / th_x[None]
    assert np.max(np.abs(th - th_x)) <= 4 * np.spacing(2.0)
    assert np.max(np.abs(u - u_x)) <= 1e-14 * np.max(np.abs(u_x))
    gcoef = -p["s1"] / (p["cs2"] / p["c"] ** 2 * dx)  # grad theta = -s1 J / (sigma dx), Sec. III.C
    assert np.max(np.abs(g - gcoef * J_x)) <= 1e-14 * np.max(np.abs(gcoef * J_x))
    # the state sum (Eq. (conseved-moment)): theta_ref per node plus every stored value, the floats of each
    # 16-byte vector summed on the integer pipes and the vector sums added in FP64
    nodes = int(np.prod(shape))
    total = s.sum_theta()
    exact = math.fsum([2.0 * nodes] + [float(v) for v in vals.ravel()])
    assert abs(total - exact) <= 1e-14 * (2.0 * nodes + float(np.sum(np.abs(vals.astype(np.float64)))))
    s.close()
