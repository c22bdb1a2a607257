"""The allocation-free norm reduction (lb_reduce_static) against lb_reduce.

lb_reduce_static serves callers that cannot call cudaMalloc (a framework
that owns all device memory, a fixed memory budget, code that must not
synchronise on an allocation): its partial sums live in a static device
array instead of a context.  Two calls in a row, on different inputs, must
each agree with the context-based lb_reduce to the 1e-12 tolerance the
other norm tests use; the second call also shows that what the first left
in the shared array does not leak into it.  This file is collected last.
"""
import numpy as np
import pytest
import torch

from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fields(d, N, seed):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.1, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2 * dx * dx / nu
    s = lb.Solver(d, N, nu, dx, dt)
    s.set_theta0(torch.from_numpy(prob.theta(N, dx)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda())
    s.step(7)
    th, _, u = s.macros()
    rng = np.random.default_rng(seed)
    ex_t = th + torch.from_numpy(rng.normal(0, 1e-3, size=tuple(th.shape))).cuda()
    ex_u = u + torch.from_numpy(rng.normal(0, 1e-4, size=tuple(u.shape))).cuda()
    return s, th, u, ex_t, ex_u


def test_static_reduce_matches_lb_reduce_on_two_calls_in_a_row():
    for d, N, seed in ((3, (40, 17, 9), 4), (2, (96, 50), 3)):
        s, th, u, ex_t, ex_u = _fields(d, N, seed)
        ref = s.reduce(th, u, ex_t, ex_u)
        want = []
        for v in ["theta"] + ["u%d" % a for a in range(d)]:
            want += [ref[v]["rmse"], ref[v]["linf"], ref[v]["rel_l2"]]
        want.append(ref["sum_theta"])
        out = torch.full((3 * (d + 1) + 1,), float("nan"), dtype=torch.float64, device="cuda")
        lb.lb_reduce_static(d, th.numel(), th, u, ex_t, ex_u, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=0.0), (d, got, want)
        s.close()


def test_static_reduce_rejects_sizes_beyond_its_maximum():
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    for d, nodes in ((2, (1 << 31) + 1), (4, 4), (2, 0)):
        with pytest.raises(lb.LBError) as ei:
            lb.lb_reduce_static(d, nodes, x, None, x, None, out)
        assert ei.value.status == lb.LB_EINVAL
