"""Pins of the oracle's wall model (walls with zero normal velocity, the
paper's Example 1 of Sec. V): the periodic scheme on the grid doubled by even
reflection, restricted to the original nodes.

What fixes it independently of the oracle:
* Example 1's exact solution (a Bessel-coefficient cosine series) is checked
  against scipy's Bessel functions and against the diffusion equation and
  the wall condition themselves;
* the errors against that solution fall at fourth order and stay within a
  factor 4 of every cell of Table 1 (the paper does not state its wall
  treatment, so digits are not expected to agree);
* a 2D problem with walls on x and periodic y converges at fourth order to
  its closed form;
* the doubled solution stays even (a lattice not closed under reflection,
  or a collision that does not commute with it, would break that), the
  normal velocity vanishes on wall nodes, and the wall-weighted total is
  conserved.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_02825_gb300 import workloads as W


def _run_mirror(case, mirror):
    m = O.MirrorModel(case.d, case.N, mirror, case.nu, case.dx, case.dt)
    p = case.problem
    f = m.run(m.initialize(p.theta(case.N, case.dx), p.grad(case.N, case.dx)), case.nsteps)
    return m, f


def test_bessel_coefficients_match_scipy():
    special = pytest.importorskip("scipy.special")
    for nu in (1.0 / 32, 1.0 / 16, 0.125, 0.01):
        z = 1.0 / (2 * math.pi * nu)
        a = W.bessel_i_all(z, 40)
        ref = special.iv(np.arange(41), z)
        assert np.max(np.abs(a - ref)) <= 1e-15 * ref[0] * 8


def test_wall_bessel_solution_solves_diffusion_with_walls():
    """theta_t = nu theta_xx (central difference in t, fourth-order central
    difference in x) and theta_x = 0 at both walls, for the series at t = 0.5."""
    p = W.WallBesselProblem(1.0 / 32)
    n, h, t = 2001, 1e-4, 0.5
    dx = 1.0 / (n - 1)
    tt = (p.theta((n,), dx, t + h) - p.theta((n,), dx, t - h)) / (2 * h)
    th = p.theta((n,), dx, t)
    lap = (-th[4:] + 16 * th[3:-1] - 30 * th[2:-2] + 16 * th[1:-3] - th[:-4]) / (12 * dx * dx)
    assert np.max(np.abs(tt[2:-2] - p.nu * lap)) <= 1e-6 * np.max(np.abs(tt))
    g = p.grad((n,), dx, t)[0]
    assert abs(g[0]) <= 1e-12 * np.max(np.abs(g)) and abs(g[-1]) <= 1e-12 * np.max(np.abs(g))
    # u(x, 0) = sin(pi x) is the initial condition of Example 1
    x = dx * np.arange(n)
    assert np.max(np.abs(p.u((n,), dx, 0.0)[0] - np.sin(np.pi * x))) <= 1e-14


@pytest.mark.parametrize("eps", [0.5, 2.0])
def test_example1_fourth_order_and_table1_magnitude(golden, eps):
    cells = {(float(r[0]), int(r[1]), r[2]): float(r[3]) for r in golden("paper_table1_1d.txt")}
    errs = {"theta": [], "u": []}
    for level in range(4):
        case = W.wall_example1(eps, level)
        m, f = _run_mirror(case, (True,))
        th, _, u = m.recover(f)
        T = case.t_end
        errs["theta"].append(O.rmse(th, case.problem.theta(case.N, case.dx, T)))
        errs["u"].append(O.rmse(u[0], case.problem.u(case.N, case.dx, T)[0]))
    for var, e in errs.items():
        rates = [math.log2(e[i] / e[i + 1]) for i in range(3)]
        assert all(3.7 <= r <= 4.5 for r in rates), (var, rates)
        assert abs(rates[-1] - 4.0) <= 0.1, (var, rates)
        for level in range(4):
            ratio = e[level] / cells[(eps, level, var)]
            assert 0.25 <= ratio <= 4.0, (var, level, ratio)


def test_mirror_solution_even_and_zero_normal_velocity():
    """2D, walls on x (17 nodes), periodic y (12 nodes), a field that is not
    itself symmetric in y: the doubled-grid solution stays even in x."""
    N, nu, dx = (17, 12), 0.03, 1.0 / 16
    dt = 0.2 * dx * dx / nu
    prob = W.ProductWaveProblem(2, nu, (1, 2), ("cos", "sin"), 2.0, 1.0)
    th0 = prob.theta(N, dx) + 0.05 * np.cos(np.pi * W.grid(N, dx)[0] * 2) * np.cos(2 * np.pi * W.grid(N, dx)[1])
    m = O.MirrorModel(2, N, (True, False), nu, dx, dt)
    f = m.run(m.initialize(th0), 25)
    thf, _, uf = m.full.recover(f)
    n0 = 2 * (N[0] - 1)
    refl = (-np.arange(n0)) % n0
    assert np.max(np.abs(thf - thf[:, refl])) <= 1e-14 * np.max(np.abs(thf))
    assert np.max(np.abs(uf[0] + uf[0][:, refl])) <= 1e-14 * np.max(np.abs(uf))
    th, _, u = m.recover(f)
    assert np.max(np.abs(u[0][:, [0, -1]])) <= 1e-13 * np.max(np.abs(u))


def test_mirror_2d_mixed_fourth_order():
    """theta = 2 + e^{-5 pi^2 nu t} cos(pi x) sin(2 pi y): walls on x at 0 and
    1, periodic y; errors fall at fourth order."""
    nu, eps = 0.02, 0.2
    errs = []
    for n in (32, 64, 128):
        dx = 1.0 / n
        dt = eps * dx * dx / nu
        N = (n + 1, n)
        prob = W.ProductWaveProblem(2, nu, (1, 2), ("cos", "sin"), 2.0, 1.0)
        steps = int(round(0.05 / dt))
        m = O.MirrorModel(2, N, (True, False), nu, dx, dt)
        f = m.run(m.initialize(prob.theta(N, dx), prob.grad(N, dx)), steps)
        _, _, u = m.recover(f)
        errs.append(O.rmse(u, prob.u(N, dx, steps * dt)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.7 <= r <= 4.4 for r in rates), rates


def test_mirror_weighted_total_conserved():
    N, nu, dx = (9, 7, 5), 0.02, 0.1
    dt = 0.15 * dx * dx / nu
    rng = np.random.default_rng(5)
    th0 = 1.5 + 0.1 * rng.standard_normal(tuple(reversed(N)))
    m = O.MirrorModel(3, N, (True, False, True), nu, dx, dt)
    f = m.initialize(th0)
    w = m.wall_weights()
    t0 = m.total(f)
    assert abs(t0 - float(np.sum(w * th0))) <= 1e-13 * t0
    f = m.run(f, 13)
    th, _, _ = m.recover(f)
    assert abs(m.total(f) - t0) <= 1e-13 * t0
    assert abs(float(np.sum(w * th)) - t0) <= 1e-13 * t0
