"""Failure detection without a GPU fault: a device-side wait that can never
complete gives up at its time bound and is reported as LB_ETIMEOUT, and the
device stays usable afterwards."""
import numpy as np
import pytest
import torch

from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_staging_wait_times_out_and_device_stays_usable():
    st, waited = lb.lb_selftest_staging_timeout(0.05)
    assert st == lb.LB_ETIMEOUT
    assert 0.04 <= waited < 2.0
    case = W.sine_2d(64)
    s = lb.Solver(2, case.N, case.nu, case.dx, case.dt)
    s.set_theta0(torch.from_numpy(case.problem.theta(case.N, case.dx)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(case.problem.grad(case.N, case.dx))).cuda())
    s.step(3)
    th, _, u = s.macros()
    ex = torch.from_numpy(case.problem.theta(case.N, case.dx, 3 * case.dt)).cuda()
    exu = torch.from_numpy(np.ascontiguousarray(case.problem.u(case.N, case.dx, 3 * case.dt))).cuda()
    r = s.reduce(th, u, ex, exu)
    assert r["theta"]["rmse"] < 1e-5


def test_selftest_rejects_unbounded_requests():
    st, _ = lb.lb_selftest_staging_timeout(100.0)
    assert st == lb.LB_EINVAL
