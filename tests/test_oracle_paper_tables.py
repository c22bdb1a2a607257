"""Oracle pins: the RMSE values the paper prints for its periodic examples.

Tables 2 (D2Q9), 3 (D3Q19) and 4 (D4Q33) are reproduced by running the
oracle on the paper's own examples (Sec. IV).  The RMSE is taken over the
closed node set j = 0..N per axis (the periodic end point counted twice).
Under that reading every printed digit of Tables 3 and 4 and of the theta
rows of Table 2 is reproduced; the u rows of Table 2 agree to within 1%.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_02825_gb300 import workloads as W


def closed(a):
    return np.pad(a, [(0, 1)] * a.ndim, mode="wrap")


def _run_case(case):
    m = O.Model(case.d, case.N, case.nu, case.dx, case.dt)
    f = m.initialize(case.problem.theta(case.N, case.dx), case.problem.grad(case.N, case.dx))
    th, _, u = m.recover(m.run(f, case.nsteps))
    T = case.t_end
    return th, u, case.problem.theta(case.N, case.dx, T), case.problem.u(case.N, case.dx, T)


def _cells(golden, name):
    out = {}
    for eps, lev, var, val in golden(name):
        out.setdefault((float(eps), lev), {})[var] = float(val)
    return out


@pytest.mark.parametrize("eps,level", [(e, l) for e in (0.1, 0.2, 0.3, 0.4) for l in (0, 1)])
def test_table2_example2(golden, eps, level):
    cells = _cells(golden, "paper_table2_2d.txt")[(eps, str(level))]
    th, u, the, ue = _run_case(W.paper_example(2, eps, level))
    got = {"theta": O.rmse(closed(th), closed(the)),
           "u_x": O.rmse(closed(u[0]), closed(ue[0])), "u_y": O.rmse(closed(u[1]), closed(ue[1]))}
    assert got["theta"] == pytest.approx(cells["theta"], rel=1e-4)
    for v in ("u_x", "u_y"):
        assert got[v] == pytest.approx(cells[v], rel=1e-2)


@pytest.mark.parametrize("eps,level", [(0.05, 0), (0.10, 0), (0.15, 0), (0.20, 0), (0.05, 1)])
def test_table3_example3(golden, eps, level):
    cells = _cells(golden, "paper_table3_3d.txt")[(eps, str(level))]
    th, u, the, ue = _run_case(W.paper_example(3, eps, level))
    got = {"theta": O.rmse(closed(th), closed(the))}
    for a, v in enumerate(("u_x", "u_y", "u_z")):
        got[v] = O.rmse(closed(u[a]), closed(ue[a]))
    for v, want in cells.items():
        assert got[v] == pytest.approx(want, rel=1e-4), v


@pytest.mark.parametrize("eps", [0.08, 0.10])
def test_table4_example4(golden, eps):
    cells = {}
    for e, t, var, val in golden("paper_table4_4d.txt"):
        if float(e) == eps:
            cells[var] = float(val)
    dx, dt = 1.0 / 10, 1.0 / 40
    nu = eps * dx * dx / dt
    N = (20,) * 4
    steps = 40
    prob = W.ProductSineProblem(4, nu, (1, 2, 3, 4), 2.0, 2.0, origin=-1.0)
    m = O.Model(4, N, nu, dx, dt)
    th, _, u = m.recover(m.run(m.initialize(prob.theta(N, dx), prob.grad(N, dx)), steps))
    T = steps * dt
    assert math.isclose(T, 1.0)
    got = {"theta": O.rmse(closed(th), closed(prob.theta(N, dx, T)))}
    ue = prob.u(N, dx, T)
    for a in range(4):
        got["u_x%d" % (a + 1)] = O.rmse(closed(u[a]), closed(ue[a]))
    for v, want in cells.items():
        assert got[v] == pytest.approx(want, rel=1e-4), v
