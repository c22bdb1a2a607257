"""Oracle pins: fourth-order convergence against closed-form Cole-Hopf solutions.

Under diffusive refinement (dx -> dx/2, dt -> dt/4, eps fixed) the RMSE of
theta and u must fall by 2^4 (Theorem 2).  A plausible slip anywhere in the
update (a wrong weight, relaxation rate, sign, or the non-equilibrium part
of the initialisation) drops the rate to 2 or destroys convergence.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_02825_gb300 import workloads as W


def _errors(case, grad0=True):
    m = O.Model(case.d, case.N, case.nu, case.dx, case.dt)
    th0 = case.problem.theta(case.N, case.dx)
    g0 = case.problem.grad(case.N, case.dx) if grad0 else np.zeros((case.d,) + th0.shape)
    th, _, u = m.recover(m.run(m.initialize(th0, g0), case.nsteps))
    T = case.t_end
    return O.rmse(th, case.problem.theta(case.N, case.dx, T)), O.rmse(u, case.problem.u(case.N, case.dx, T))


def _rates(family, Ns, **kw):
    errs = [_errors(family(N), **kw) for N in Ns]
    return [(np.log2(a[0] / b[0]), np.log2(a[1] / b[1])) for a, b in zip(errs, errs[1:])]


def test_1d_sine_fourth_order():
    for cr_t, cr_u in _rates(W.sine_1d, (16, 32, 64, 128)):
        assert abs(cr_t - 4) < 0.1 and abs(cr_u - 4) < 0.1


def test_2d_sine_fourth_order():
    for cr_t, cr_u in _rates(W.sine_2d, (32, 64, 128, 256)):
        assert abs(cr_t - 4) < 0.1 and abs(cr_u - 4) < 0.1


def test_3d_fourier_fourth_order():
    (cr_t, cr_u), = _rates(W.fourier_3d, (32, 64))
    assert abs(cr_t - 4) < 0.2
    assert cr_u > 3.8


def test_equilibrium_only_init_is_second_order():
    """Dropping the non-equilibrium initial term (Sec. IV, Eq. (f-feq-o5)) makes
    the scheme second order: the convergence pins detect that omission."""
    rates = _rates(W.sine_2d, (32, 64, 128), grad0=False)
    assert all(abs(cr_u - 2) < 0.3 for _, cr_u in rates)
