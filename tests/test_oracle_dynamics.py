"""Oracle pins: the collision, streaming, conservation and recovery.

The expected values come from the paper's definitions written out here
independently of the oracle's matrices: moment sums over the velocity list,
the diagonal relaxation S and the equilibrium moments of Eq. (feq).
"""
import itertools

import numpy as np
import pytest

import oracle as O


def _moment_sums(e, f):
    """theta, J_a, P_ab, third-order and fourth-order moment sums of one node."""
    d = e.shape[1]
    th = f.sum()
    J = e.T @ f
    P = np.einsum("ia,ib,i->ab", e, e, f)
    pairs = list(itertools.combinations(range(d), 2))
    T = np.array([np.sum(e[:, a] * e[:, b] ** 2 * f) for a, b in pairs]
                 + [np.sum(e[:, a] ** 2 * e[:, b] * f) for a, b in pairs])
    F = np.array([np.sum(e[:, a] ** 2 * e[:, b] ** 2 * f) for a, b in pairs])
    return th, J, P, T, F


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_single_node_collision_relaxes_each_moment(d):
    """On a 1-node periodic grid streaming is the identity, so one step is one
    collision: m* = m - S (m - m^eq) with m^eq = M w theta (Eq. (distribution-f))."""
    rng = np.random.default_rng(1)
    eps = 0.13
    m = O.Model(d, [1] * d, eps, 1.0, 1.0)
    p = m.params
    e = O.lattice(d).astype(float)
    w = O.weights(d, p["w1"], p["wd"])
    f = rng.uniform(0.0, 1.0, size=m.q)
    out = m.step(f.reshape((m.q,) + (1,) * d)).ravel()
    th, J, P, T, F = _moment_sums(e, f)
    th2, J2, P2, T2, F2 = _moment_sums(e, out)
    sigma = 2 * p["w1"] + 4 * (d - 1) * p["wd"]
    assert abs(th2 - th) < 1e-14
    assert np.allclose(J2, (1 - p["s1"]) * J, atol=1e-14)
    for a in range(d):
        assert abs(P2[a, a] - (P[a, a] - p["s2x"] * (P[a, a] - sigma * th))) < 1e-14
        for b in range(a + 1, d):
            assert abs(P2[a, b] - (1 - p["s22"]) * P[a, b]) < 1e-14
    # rate-1 moments land on equilibrium: third order 0, fourth order 4 w_d theta
    assert np.allclose(T2, 0.0, atol=1e-14)
    assert np.allclose(F2, 4 * p["wd"] * th, atol=1e-14)
    assert abs(sum(w) - 1) < 4e-15


@pytest.mark.parametrize("d", [1, 2, 3])
def test_streaming_moves_population_i_by_e_i(d):
    """A unit pulse in population i at x0: after one step population k sits only
    at x0 + e_k (periodic), and the total is conserved."""
    N = [5] * d
    m = O.Model(d, N, 0.02, 0.2, 0.2 * 0.2)
    e = O.lattice(d)
    x0 = [1, 3, 2, 4][:d]
    for i in range(m.q):
        f = np.zeros((m.q,) + tuple(reversed(N)))
        f[(i,) + tuple(reversed(x0))] = 1.0
        out = m.step(f)
        assert abs(out.sum() - 1.0) < 1e-14
        for k in range(m.q):
            dest = [(x0[a] + e[k, a]) % N[a] for a in range(d)]
            mask = np.ones(tuple(reversed(N)), dtype=bool)
            mask[tuple(reversed(dest))] = False
            assert np.all(out[k][mask] == 0.0)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_uniform_theta_is_a_fixed_point(d):
    N = [6] * d
    m = O.Model(d, N, 0.02, 1.0 / 6, 0.01)
    th0 = np.full(tuple(reversed(N)), 1.7)
    f = m.initialize(th0, np.zeros((d,) + th0.shape))
    assert np.allclose(f, m.matrices()["w"].reshape((-1,) + (1,) * d) * 1.7, atol=1e-15)
    f2 = m.run(f, 7)
    assert np.allclose(f2, f, atol=1e-15)
    th, g, u = m.recover(f2)
    assert np.allclose(th, 1.7, atol=1e-15)
    assert np.allclose(u, 0.0, atol=1e-15) and np.allclose(g, 0.0, atol=1e-13)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_total_theta_is_conserved(d):
    """m0 is collision invariant and streaming permutes values, so sum theta is
    constant on a periodic grid."""
    rng = np.random.default_rng(7 + d)
    N = [7, 5, 4][:d]
    m = O.Model(d, N, 0.02, 1.0 / 7, 0.01)
    f = rng.uniform(0.1, 1.0, size=(m.q,) + tuple(reversed(N)))
    s0 = m.total(f)
    f2 = m.run(f, 50)
    th, _, _ = m.recover(f2)
    assert abs(m.total(f2) - s0) <= 1e-13 * s0
    assert abs(th.sum() - s0) <= 1e-13 * s0


@pytest.mark.parametrize("d", [1, 2, 3])
def test_init_first_moment_reproduces_gradient(d):
    """Init from Eq. (f-feq-o5): sum_k c_k f^ne_k = -(dt/s1) c_s^2 grad theta0,
    so the recovery returns grad theta0 and u = -2 nu grad theta0 / theta0
    exactly (the paper's identity below Eq. (f-feq-o5))."""
    rng = np.random.default_rng(3)
    N = [6, 5, 4][:d]
    m = O.Model(d, N, 0.03, 0.1, 0.02)
    th0 = rng.uniform(1.0, 2.0, size=tuple(reversed(N)))
    g0 = rng.normal(size=(d,) + th0.shape)
    f = m.initialize(th0, g0)
    th, g, u = m.recover(f)
    assert np.allclose(th, th0, atol=1e-14)
    assert np.allclose(g, g0, atol=1e-12)
    assert np.allclose(u, -2 * m.params["nu"] * g0 / th0[None], atol=1e-13)


def test_fd_gradient_used_when_none_given():
    N = [8, 8]
    m = O.Model(2, N, 0.03, 0.125, 0.02)
    rng = np.random.default_rng(4)
    th0 = rng.uniform(1.0, 2.0, size=(8, 8))
    assert np.array_equal(m.initialize(th0), m.initialize(th0, m.fd4_gradient(th0)))


@pytest.mark.parametrize("d,N,n", [(1, (40,), 4), (2, (30, 22), 3), (3, (14, 12, 11), 2)])
def test_patch_of_side_2n_plus_3_reproduces_the_full_grid(d, N, n):
    """The full-size GPU tests sample nodes by running the oracle on a small
    periodic patch: after n steps a node only sees the initial data within
    Chebyshev distance n.  Check that argument on the oracle itself."""
    from paper_2309_02825_gb300 import workloads as W
    from tests.test_gpu_fullsize import _patch

    prob = W.FourierProblem.random(d, 0.02, 6, 3, 0.1, 1.5, 5)
    dx = 1.0 / max(N)
    dt = 0.2 * dx * dx / 0.02
    th0, g0 = prob.theta(N, dx), prob.grad(N, dx)
    full = O.Model(d, N, 0.02, dx, dt)
    th, _, u = full.recover(full.run(full.initialize(th0, g0), n))
    half = n + 1
    pm = O.Model(d, [2 * half + 1] * d, 0.02, dx, dt)
    rng = np.random.default_rng(0)
    for _ in range(6):
        c = tuple(int(rng.integers(0, k)) for k in N)
        pt, pg = _patch(th0, c, half), _patch(g0, c, half)
        tho, _, uo = pm.recover(pm.run(pm.initialize(pt, pg), n))
        mid = (half,) * d
        assert abs(tho[mid] - th[tuple(reversed(c))]) < 1e-14
        assert np.allclose(uo[(slice(None),) + mid], u[(slice(None),) + tuple(reversed(c))], atol=1e-15, rtol=0)
