"""The fixed-point collision product (64-bit state value times a constant
with 64 fraction bits, rounded to nearest with ties upward) against exact
integer arithmetic: the split-word form the LB_FX64 collisions use and the
128-bit form, bit for bit, over the whole admitted range
(|k| <= 2^63 - 2^34, |a| < 2^63 - 2^31), including ties, the ends of the
range and values whose low words have the sign bit set; plus the host's
rejection of relaxation sets whose constants leave (-1/2, 1/2)."""
import numpy as np
import pytest
import torch

from paper_2309_02825_gb300 import lb

pytestmark = pytest.mark.gpu

A_MAX = 2 ** 63 - 2 ** 31  # exclusive
K_MAX = 2 ** 63 - 2 ** 34  # inclusive


def _exact(a, k):
    return (a * k + 2 ** 63) >> 64  # Python integers: exact, floor division


def _cases(rng):
    a_edge = [0, 1, -1, 2 ** 31 - 1, 2 ** 31, -(2 ** 31), -(2 ** 31) - 1, 2 ** 32 - 1, 2 ** 32, -(2 ** 32),
              2 ** 61 - 1, 2 ** 61, -(2 ** 61), 2 ** 62, -(2 ** 62), A_MAX - 1, -(A_MAX - 1), -A_MAX,
              (2 ** 31 - 1) << 32, ((2 ** 31 - 1) << 32) - 1, 0x7FFFFFFE80000000 - 1]
    k_edge = [0, 1, -1, 2 ** 31 - 1, 2 ** 31, -(2 ** 31), 2 ** 32 - 1, 2 ** 32 + 2 ** 31, K_MAX, -K_MAX, K_MAX - 1,
              -K_MAX + 2 ** 31, 2 ** 62, -(2 ** 62), 2 ** 61 + 2 ** 31 - 1, K_MAX - 2 ** 31, -(K_MAX - 2 ** 31 - 1)]
    pairs = [(a, k) for a in a_edge for k in k_edge]
    for _ in range(60000):
        ba, bk = int(rng.integers(1, 64)), int(rng.integers(1, 64))
        a = int(rng.integers(0, 2 ** 62)) << 2 | int(rng.integers(0, 4))
        k = int(rng.integers(0, 2 ** 62)) << 2 | int(rng.integers(0, 4))
        a &= (1 << ba) - 1
        k &= (1 << bk) - 1
        a = -a if rng.random() < 0.5 else a
        k = -k if rng.random() < 0.5 else k
        pairs.append((a, k))
    # exact ties: a k / 2^64 has a fractional part of exactly 1/2 when
    # k = 2^s and a = (2j + 1) 2^(63 - s)
    for s in range(1, 63):
        k = 1 << s
        for _ in range(20):
            j = int(rng.integers(0, 2 ** min(s, 40)))
            a = (2 * j + 1) << (63 - s)
            if abs(a) < A_MAX:
                pairs.append((a, k))
                pairs.append((-a, k))
                pairs.append((a, -k))
    return [(a, k) for a, k in pairs if -A_MAX < a < A_MAX and -K_MAX <= k <= K_MAX]


def test_split_product_is_exact():
    rng = np.random.default_rng(31)
    pairs = _cases(rng)
    a = torch.tensor([p[0] for p in pairs], dtype=torch.int64).cuda()
    k = torch.tensor([p[1] for p in pairs], dtype=torch.int64).cuda()
    split, wide = lb.lb_selftest_mulfx(a, k)
    want = np.array([_exact(x, y) for x, y in pairs], dtype=object)
    got_s = split.cpu().numpy().astype(object)
    got_w = wide.cpu().numpy().astype(object)
    bad = [i for i in range(len(pairs)) if got_s[i] != want[i]]
    assert not bad, [(pairs[i], got_s[i], want[i]) for i in bad[:5]]
    bad = [i for i in range(len(pairs)) if got_w[i] != want[i]]
    assert not bad, [(pairs[i], got_w[i], want[i]) for i in bad[:5]]


def test_selftest_argument_errors():
    lib = lb.load()
    assert lib.lb_selftest_mulfx(None, None, -1, None, None, None) == lb.LB_EINVAL
    assert lib.lb_selftest_mulfx(None, None, 3, None, None, None) == lb.LB_EINVAL
    assert lib.lb_selftest_mulfx(None, None, 0, None, None, None) == lb.LB_OK


@pytest.mark.parametrize("d,eps_ok,eps_bad", [(2, 1.6, 1.7), (3, 0.85, 0.9), (4, 0.6, 0.62)])
def test_fx64_rejects_constants_outside_half_interval(d, eps_ok, eps_bad):
    """The paper's set keeps every fixed-point collision constant inside
    (-1/2, 1/2) up to eps = 1.66 (2D), 0.88 (3D), 0.61 (4D); beyond it cA
    leaves the range of the collision product and LB_FX64 is refused (FP64
    still accepts it)."""
    N, dx, dt = (4,) * d, 0.1, 0.1
    lb.Solver(d, N, eps_ok * dx * dx / dt, dx, dt, precision="fx64").close()
    with pytest.raises(lb.LBError) as ei:
        lb.Solver(d, N, eps_bad * dx * dx / dt, dx, dt, precision="fx64")
    assert ei.value.status == lb.LB_EINVAL
    lb.Solver(d, N, eps_bad * dx * dx / dt, dx, dt, precision="fp64").close()
    s = lb.Solver(d, N, eps_ok * dx * dx / dt, dx, dt, precision="fx64")
    with pytest.raises(lb.LBError) as ei:
        s.set_viscosity(eps_bad * dx * dx / dt)
    assert ei.value.status == lb.LB_EINVAL
    s.close()


def test_fx64_batch_refuses_an_instance_outside_the_range():
    """lb_batch_create applies the same rule per instance."""
    dx, dt = 0.1, 0.1
    nus = [0.2 * dx * dx / dt, 1.7 * dx * dx / dt]  # eps = 0.2 and 1.7 (2D limit 1.66)
    with pytest.raises(lb.LBError) as ei:
        lb.Batch([(8, 8), (8, 8)], nus, [dx, dx], [dt, dt], precision="fx64")
    assert ei.value.status == lb.LB_EINVAL
    lb.Batch([(8, 8), (8, 8)], nus, [dx, dx], [dt, dt], precision="fp64").close()
    lb.Batch([(8, 8)], nus[:1], [dx], [dt], precision="fx64").close()
