"""GPU parity at the full benchmark sizes (2D 4096^2, 3D 256^3), on sampled nodes.

After n steps the pre-collision f at a node depends only on the initial
data within Chebyshev distance n (one lattice link per step), and the
initialisation with an analytic gradient is local.  So the oracle, run on a
periodic patch of side 2n + 3 centred on a sampled node, reproduces that
node exactly: whatever crosses the patch's own wrap needs more than n steps
to reach the centre.  The solver runs through the same C-ABI calls and launch
configuration that bench.py times.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _patch(field, center, half):
    """Periodic patch of side 2*half+1 around `center` (x first) of a field
    with shape (N_{d-1}, ..., N_0), optionally with a leading component axis."""
    d = len(center)
    idx = [np.arange(c - half, c + half + 1) for c in center]
    lead = field.ndim - d
    out = field
    for a in range(d):
        ax = lead + (d - 1 - a)
        out = np.take(out, idx[a] % field.shape[ax], axis=ax)
    return out


def _samples(N, rng, k=24):
    d = len(N)
    pts = [tuple(0 for _ in N), tuple(n - 1 for n in N), tuple([63] + [0] * (d - 1)),
           tuple([64] + [n - 1 for n in N[1:]]), tuple([N[0] - 1] + [n // 2 for n in N[1:]])]
    while len(pts) < k:
        pts.append(tuple(int(rng.integers(0, n)) for n in N))
    return [tuple(v % n for v, n in zip(p, N)) for p in pts]  # warp-edge points wrap on short rows


def _check(case, precision, nsteps, theta_ref=0.0):
    N, d = case.N, case.d
    th0 = case.problem.theta(N, case.dx)
    g0 = np.ascontiguousarray(case.problem.grad(N, case.dx))
    s = lb.Solver(d, N, case.nu, case.dx, case.dt, precision=precision, theta_ref=theta_ref)
    s.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    s.step(nsteps)
    th, gr, u = s.macros()
    total = s.sum_theta()
    th, u = th.cpu().numpy(), u.cpu().numpy()
    s.close()
    half = nsteps + 1
    P = 2 * half + 1
    m = O.Model(d, [P] * d, case.nu, case.dx, case.dt)
    rng = np.random.default_rng(99)
    worst = {"theta": 0.0, "u": 0.0}
    # normwise: differences relative to the field's global maximum
    scale_t, scale_u = float(np.max(np.abs(th))), float(np.max(np.abs(u)))
    for c in _samples(N, rng):
        pt = _patch(th0, c, half)
        pg = _patch(g0, c, half)
        tho, _, uo = m.recover(m.run(m.initialize(pt, pg), nsteps))
        mid = (half,) * d
        got_t = th[tuple(reversed(c))]
        got_u = u[(slice(None),) + tuple(reversed(c))]
        worst["theta"] = max(worst["theta"], abs(got_t - tho[mid]) / scale_t)
        worst["u"] = max(worst["u"], float(np.max(np.abs(got_u - uo[(slice(None),) + mid])) / scale_u))
    return worst, total, float(th0.sum())


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_fullsize_2d_4096(precision):
    worst, total, t0 = _check(W.sine_2d(4096), precision, 3)
    assert worst["theta"] <= 1e-12 and worst["u"] <= 1e-12, worst
    assert abs(total - t0) <= 1e-13 * t0


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_fullsize_3d_256(precision):
    worst, total, t0 = _check(W.fourier_3d(256), precision, 3)
    assert worst["theta"] <= 1e-12 and worst["u"] <= 1e-12, worst
    assert abs(total - t0) <= 1e-13 * t0


@pytest.mark.parametrize("case,ref", [(lambda: W.sine_2d(4096), 2.0), (lambda: W.fourier_3d(256), 1.5)])
def test_fullsize_fp32_shifted(case, ref):
    c = case()
    worst, total, t0 = _check(c, "fp32s", 3, theta_ref=ref)
    # stored values are O(1): float rounding of a handful of operations per step
    assert worst["theta"] <= 1e-6 and worst["u"] <= 1e-4, worst
    assert abs(total - t0) <= 1e-6 * t0


def _mirror_index(k, n):
    """Node of the evenly doubled axis (period 2(n-1)) folded back into
    0..n-1, and the sign of the wall-normal gradient component there."""
    p = 2 * (n - 1)
    j = np.mod(k, p)
    refl = j > n - 1
    return np.where(refl, p - j, j), np.where(refl, -1.0, 1.0)


def _patch_walls(field, center, half, mirror, vector=False):
    """Patch of side 2*half+1 around `center` on the grid doubled by even
    reflection across the walls of each mirror axis (periodic elsewhere);
    for a vector field the wall-normal component is odd (zero on the wall)."""
    d = len(center)
    lead = 1 if vector else 0
    out = np.array(field, dtype=np.float64)
    if vector:
        for a in range(d):
            if mirror[a]:
                n = field.shape[lead + d - 1 - a]
                sl = [slice(None)] * out.ndim
                sl[0] = a
                for j in (0, n - 1):
                    sl[lead + d - 1 - a] = j
                    out[tuple(sl)] = 0.0
    for a in range(d):
        ax = lead + (d - 1 - a)
        n = field.shape[ax]
        k = np.arange(center[a] - half, center[a] + half + 1)
        if mirror[a]:
            idx, sgn = _mirror_index(k, n)
            out = np.take(out, idx, axis=ax)
            if vector:
                shape = [1] * out.ndim
                shape[ax] = len(k)
                out[a] = out[a] * sgn.reshape(shape[1:])
        else:
            out = np.take(out, k % n, axis=ax)
    return out


def _check_walls(case, mirror, precision, nsteps):
    N, d = case.N, case.d
    th0 = case.problem.theta(N, case.dx)
    g0 = np.ascontiguousarray(case.problem.grad(N, case.dx))
    kinds = ["mirror" if m else "periodic" for m in mirror]
    s = lb.Solver(d, N, case.nu, case.dx, case.dt, precision=precision, boundary=kinds)
    s.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    s.step(nsteps)
    th, _, u = s.macros()
    th, u = th.cpu().numpy(), u.cpu().numpy()
    s.close()
    half = nsteps + 1
    P = 2 * half + 1
    m = O.Model(d, [P] * d, case.nu, case.dx, case.dt)
    rng = np.random.default_rng(98)
    worst = {"theta": 0.0, "u": 0.0}
    scale_t, scale_u = float(np.max(np.abs(th))), float(np.max(np.abs(u)))
    pts = _samples(N, rng) + [tuple([1] + [n - 2 for n in N[1:]]), tuple([N[0] - 2] + [1] * (d - 1))]
    for c in pts:
        pt = _patch_walls(th0, c, half, mirror)
        pg = _patch_walls(g0, c, half, mirror, vector=True)
        tho, _, uo = m.recover(m.run(m.initialize(pt, pg), nsteps))
        mid = (half,) * d
        got_t = th[tuple(reversed(c))]
        got_u = u[(slice(None),) + tuple(reversed(c))]
        worst["theta"] = max(worst["theta"], abs(got_t - tho[mid]) / scale_t)
        worst["u"] = max(worst["u"], float(np.max(np.abs(got_u - uo[(slice(None),) + mid])) / scale_u))
    return worst


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_fullsize_2d_4096_walls(precision):
    """4096^2 with walls on both axes (corners included among the samples)."""
    worst = _check_walls(W.sine_2d(4096), (True, True), precision, 3)
    assert worst["theta"] <= 1e-12 and worst["u"] <= 1e-12, worst


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_fullsize_3d_256_walls(precision):
    """256^3 with walls on x and z, periodic y."""
    worst = _check_walls(W.fourier_3d(256), (True, False, True), precision, 2)
    assert worst["theta"] <= 1e-12 and worst["u"] <= 1e-12, worst


def test_fx64_16384_squared_offsets_beyond_2_31():
    """16384^2 D2Q9 FX64 (268 M nodes, 2 x 19.3 GB of state): population
    offsets i * slab pass 2^31 elements, so any 32-bit index arithmetic in
    the initialisation, sweep or recovery would misplace values.  Sampled
    nodes (first and last rows, last population slabs' far corners) against
    the patch oracle after 2 steps."""
    n, nsteps = 16384, 2
    case = W.sine_2d(n)
    N = case.N
    th0 = case.problem.theta(N, case.dx)
    g0 = np.ascontiguousarray(case.problem.grad(N, case.dx))
    s = lb.Solver(2, N, case.nu, case.dx, case.dt, precision="fx64")
    pitch, slab, _ = s.state_layout()
    assert int(s.params["q"]) * slab > 2 ** 31
    s.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    s.step(nsteps)
    th, _, u = s.macros(want=("theta", "u"))
    half = nsteps + 1
    m = O.Model(2, [2 * half + 1] * 2, case.nu, case.dx, case.dt)
    pts = [(0, 0), (n - 1, n - 1), (n - 1, 0), (0, n - 1), (8191, 12000), (16000, 16383), (5, 16380)]
    for c in pts:
        tho, _, uo = m.recover(m.run(m.initialize(_patch(th0, c, half), _patch(g0, c, half)), nsteps))
        got_t = float(th[c[1], c[0]].item())
        got_u = u[:, c[1], c[0]].cpu().numpy()
        assert abs(got_t - tho[half, half]) <= 1e-12 * 3.0, (c, got_t, tho[half, half])
        assert np.max(np.abs(got_u - uo[:, half, half])) <= 1e-12 * 0.3, (c, got_u, uo[:, half, half])
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_fullsize_4d_example4_50(precision):
    """The 4D benchmark case (the paper's Example 4 at dx = 1/25: 50^4 nodes,
    D4Q33, dt = 1/250) on sampled nodes against the patch oracle."""
    dx, dt, eps = 1.0 / 25, 1.0 / 250, 0.08
    nu = eps * dx * dx / dt
    prob = W.ProductSineProblem(4, nu, (1, 2, 3, 4), 2.0, 2.0, origin=-1.0)
    case = W.Case("example4_50", 4, (50,) * 4, nu, dx, dt, 250, prob)
    worst, total, t0 = _check(case, precision, 2)
    assert worst["theta"] <= 1e-12 and worst["u"] <= 1e-12, worst
    assert abs(total - t0) <= 1e-13 * t0


def test_fullsize_batched_512_instances():
    """The batched benchmark workload (512 instances, autotuned schedule, FP32
    shifted): sampled instances equal single-grid solves bit for bit after a
    recorded graph plus direct launches (the single-grid solver is itself
    checked against the oracle)."""
    cases = W.batched_2d(512, nsteps=2000)
    th0 = np.concatenate([c.problem.theta(c.N, c.dx).ravel() for c in cases])
    g0 = np.concatenate([np.ascontiguousarray(c.problem.grad(c.N, c.dx)).ravel() for c in cases])
    b = lb.Batch([c.N for c in cases], [c.nu for c in cases], [c.dx for c in cases], [c.dt for c in cases],
                 precision="fp32s", theta_ref=[1.5] * len(cases))
    b.autotune(4)
    b.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    n = 37
    b.step(n)
    th, u = b.macros()
    ths, us = b.split(th), b.split(u, 2)
    rng = np.random.default_rng(512)
    for j in sorted(set(int(v) for v in rng.integers(0, len(cases), 6)) | {0, len(cases) - 1}):
        c = cases[j]
        s = lb.Solver(2, c.N, c.nu, c.dx, c.dt, precision="fp32s", theta_ref=1.5)
        s.set_theta0(torch.from_numpy(c.problem.theta(c.N, c.dx)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(c.problem.grad(c.N, c.dx))).cuda())
        s.step(n)
        t1, _, u1 = s.macros()
        assert torch.equal(ths[j], t1), j
        assert torch.equal(us[j], u1), j
        s.close()
    b.close()
