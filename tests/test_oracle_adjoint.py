"""Oracle pin for the reference gradient: the discrete adjoint of the whole
forward map (initialisation with the FD4 gradient, T steps of
Eq. (distribution-f), recovery of u by Eq. (ui-compute), velocity misfit)
against central finite differences of the oracle's own forward loss, on 16
random theta0 directions and on nu.  A transposed operator, a dropped term
or a wrong eps-derivative of Eq. (Bur-Sol) shows up as an O(1) mismatch."""
import numpy as np
import pytest

import oracle as O
from paper_2309_02825_gb300 import workloads as W


def _case(d, N, T, seed):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.05, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2048 * dx * dx / nu
    rng = np.random.default_rng(seed + 1)
    tgt = W.FourierProblem(d, nu, prob.offset, prob.k, prob.amp + rng.normal(0, 0.01, len(prob.amp)),
                           prob.phase)
    return prob.theta(N, dx), tgt.u(N, dx, T * dt), nu, dx, dt


@pytest.mark.parametrize("d,N,T", [(1, (24,), 20), (2, (10, 8), 12), (3, (6, 5, 4), 5)])
def test_oracle_adjoint_matches_finite_differences(d, N, T):
    th0, ut, nu, dx, dt = _case(d, N, T, 31 + d)
    m = O.Model(d, N, nu, dx, dt)
    L, g, dnu = m.adjoint(th0, ut, T)
    assert L == pytest.approx(m.loss(th0, ut, T), rel=1e-14)
    rng = np.random.default_rng(d)
    for _ in range(16):
        v = rng.normal(size=th0.shape)
        h = 1e-6
        fd = (m.loss(th0 + h * v, ut, T) - m.loss(th0 - h * v, ut, T)) / (2 * h)
        assert np.sum(g * v) == pytest.approx(fd, rel=2e-6, abs=1e-12 * abs(L))
    hn = 1e-6 * nu
    fd_nu = (O.Model(d, N, nu + hn, dx, dt).loss(th0, ut, T) - O.Model(d, N, nu - hn, dx, dt).loss(th0, ut, T)) / (2 * hn)
    assert dnu == pytest.approx(fd_nu, rel=2e-6)


@pytest.mark.parametrize("d,N,T", [(1, (6,), 7), (2, (5, 4), 4)])
def test_oracle_adjoint_matches_dense_jacobian(d, N, T):
    """Exact check without finite-difference truncation: theta0 -> f_T is
    linear (initialisation with the FD4 gradient, then T linear steps), so
    its columns are forward runs of unit vectors; u = (2 - s1) c J / theta is
    then differentiated by hand, giving dL/dtheta0 to rounding."""
    th0, ut, nu, dx, dt = _case(d, N, T, 41 + d)
    m = O.Model(d, N, nu, dx, dt)
    _, g, _ = m.adjoint(th0, ut, T)
    e = m.matrices()["e"]  # (q, d) lattice velocities
    p = m.params
    ucoef = (2.0 - p["s1"]) * p["c"]

    def moments(f):
        th = f.sum(axis=0)
        J = np.stack([np.tensordot(e[:, a], f, axes=(0, 0)) for a in range(d)])
        return th, J

    fT = m.run(m.initialize(th0), T)
    th, J = moments(fT)
    u = ucoef * J / th[None]
    r = u - ut
    dense = np.zeros(th0.size)
    for j in range(th0.size):
        ej = np.zeros(th0.size)
        ej[j] = 1.0
        dth, dJ = moments(m.run(m.initialize(ej.reshape(th0.shape)), T))
        du = ucoef * (dJ * th[None] - J * dth[None]) / (th[None] ** 2)
        dense[j] = np.sum(r * du)
    assert np.max(np.abs(g.ravel() - dense)) <= 1e-12 * np.max(np.abs(dense))


@pytest.mark.parametrize("d,N,T", [(1, (16,), 12), (2, (8, 6), 8), (3, (5, 4, 4), 4)])
def test_oracle_dnu_matches_fourth_order_differences(d, N, T):
    """dL/dnu to about 1e-10: the loss is a smooth function of nu (eps enters
    the relaxation rates and weights of Eq. (Bur-Sol) rationally), so the
    five-point difference [L(-2h) - 8 L(-h) + 8 L(h) - L(2h)] / 12h has
    truncation error O(h^4) and rounding error O(eps_mach / h); at h = 3e-4 nu
    the two agree to 2e-13 .. 7e-11 on these cases.  A wrong eps-derivative
    anywhere in the adjoint (collision, initialisation or recovery term) is
    off by far more."""
    th0, ut, nu, dx, dt = _case(d, N, T, 51 + d)
    _, _, dnu = O.Model(d, N, nu, dx, dt).adjoint(th0, ut, T)
    h = 3e-4 * nu
    Lh = {k: O.Model(d, N, nu + k * h, dx, dt).loss(th0, ut, T) for k in (-2, -1, 1, 2)}
    fd4 = (Lh[-2] - 8 * Lh[-1] + 8 * Lh[1] - Lh[2]) / (12 * h)
    assert dnu == pytest.approx(fd4, rel=1e-9)
