"""The CUDA path reproduces the paper's printed RMSE tables directly.

The paper's Example 3 (D3Q19, Table 3) and Example 4 (D4Q33, Table 4), run
through the C ABI in FP64 and FX64, must give every printed digit (relative
1e-4), with the readings recorded for the oracle pins: RMSE over the closed
node set j = 0..N per axis; Example 4 with dt = 1/40 at dx = 1/10 and theta
carrying the factor 1/2."""
import numpy as np
import pytest
import torch

from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W
from tests.conftest import read_golden

pytestmark = pytest.mark.gpu


def closed(a):
    return np.pad(a, [(0, 1)] * a.ndim, mode="wrap")


def _rmse(a, b):
    return float(np.sqrt(np.mean((closed(a) - closed(b)) ** 2)))


def _run(d, N, nu, dx, dt, steps, prob, precision):
    s = lb.Solver(d, N, nu, dx, dt, precision=precision)
    s.set_theta0(torch.from_numpy(prob.theta(N, dx)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda())
    s.step(steps)
    th, _, u = s.macros()
    s.close()
    return th.cpu().numpy(), u.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("eps", [0.05, 0.10, 0.15, 0.20])
def test_table3_on_gpu(precision, eps):
    cells = {r[2]: float(r[3]) for r in read_golden("paper_table3_3d.txt") if float(r[0]) == eps and r[1] == "0"}
    c = W.paper_example(3, eps, 0)
    th, u = _run(3, c.N, c.nu, c.dx, c.dt, c.nsteps, c.problem, precision)
    T = c.t_end
    got = {"theta": _rmse(th, c.problem.theta(c.N, c.dx, T))}
    ue = c.problem.u(c.N, c.dx, T)
    for a, v in enumerate(("u_x", "u_y", "u_z")):
        got[v] = _rmse(u[a], ue[a])
    for v, want in cells.items():
        assert got[v] == pytest.approx(want, rel=1e-4), v


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("eps", [0.08, 0.10])
def test_table4_on_gpu(precision, eps):
    cells = {r[2]: float(r[3]) for r in read_golden("paper_table4_4d.txt") if float(r[0]) == eps}
    dx, dt = 1.0 / 10, 1.0 / 40
    nu = eps * dx * dx / dt
    N = (20,) * 4
    prob = W.ProductSineProblem(4, nu, (1, 2, 3, 4), 2.0, 2.0, origin=-1.0)
    th, u = _run(4, N, nu, dx, dt, 40, prob, precision)
    T = 40 * dt
    got = {"theta": _rmse(th, prob.theta(N, dx, T))}
    ue = prob.u(N, dx, T)
    for a in range(4):
        got["u_x%d" % (a + 1)] = _rmse(u[a], ue[a])
    for v, want in cells.items():
        assert got[v] == pytest.approx(want, rel=1e-4), v
