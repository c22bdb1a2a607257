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


def _loss_with_theta(m, th0, ut, tt, T):
    """L = 1/2 |u(T) - ut|^2 + 1/2 |theta(T) - tt|^2 from plain oracle runs
    (initialisation with the FD4 gradient, T steps, recovery)."""
    th, _, u = m.recover(m.run(m.initialize(th0), T))
    return 0.5 * float(np.sum((u - ut) ** 2)) + 0.5 * float(np.sum((th - tt) ** 2))


@pytest.mark.parametrize("d,N,T", [(1, (6,), 7), (2, (5, 4), 4), (3, (4, 3, 3), 3)])
def test_oracle_theta_misfit_term_matches_dense_jacobian(d, N, T):
    """The optional theta term of the loss: theta = sum_k f_k, so it seeds
    dL/df_k with theta - theta_target at every k.  Checked exactly against the
    dense Jacobian of the linear map theta0 -> f_T, and dL/dnu (theta has no
    explicit eps dependence) against a five-point difference in nu."""
    th0, ut, nu, dx, dt = _case(d, N, T, 61 + d)
    rng = np.random.default_rng(7 + d)
    tt = th0 + 0.01 * rng.standard_normal(th0.shape)
    m = O.Model(d, N, nu, dx, dt)
    L, g, dnu = m.adjoint(th0, ut, T, theta_target=tt)
    assert L == pytest.approx(_loss_with_theta(m, th0, ut, tt, T), rel=1e-13)
    e = m.matrices()["e"]
    p = m.params
    ucoef = (2.0 - p["s1"]) * p["c"]

    def moments(f):
        return f.sum(axis=0), np.stack([np.tensordot(e[:, a], f, axes=(0, 0)) for a in range(d)])

    th, J = moments(m.run(m.initialize(th0), T))
    r = ucoef * J / th[None] - ut
    rt = th - tt
    dense = np.zeros(th0.size)
    for j in range(th0.size):
        ej = np.zeros(th0.size)
        ej[j] = 1.0
        dth, dJ = moments(m.run(m.initialize(ej.reshape(th0.shape)), T))
        du = ucoef * (dJ * th[None] - J * dth[None]) / (th[None] ** 2)
        dense[j] = np.sum(r * du) + np.sum(rt * dth)
    assert np.max(np.abs(g.ravel() - dense)) <= 1e-12 * np.max(np.abs(dense))
    # the theta term is not negligible here: dropping it moves the gradient by O(1)
    _, g_u, _ = m.adjoint(th0, ut, T)
    assert np.max(np.abs(g - g_u)) > 1e-3 * np.max(np.abs(dense))
    h = 3e-4 * nu
    Lh = {k: _loss_with_theta(O.Model(d, N, nu + k * h, dx, dt), th0, ut, tt, T) for k in (-2, -1, 1, 2)}
    assert dnu == pytest.approx((Lh[-2] - 8 * Lh[-1] + 8 * Lh[1] - Lh[2]) / (12 * h), rel=1e-9)


@pytest.mark.parametrize("d,N,T", [(1, (24,), 20), (2, (10, 8), 13), (3, (6, 5, 4), 7)])
def test_oracle_checkpointed_adjoint_is_bit_identical(d, N, T):
    """Keeping every C-th forward state and recomputing one segment at a time
    replays the same steps, so the loss and both gradients equal those of the
    run that keeps every state, bit for bit (C = 1, T, and C not dividing T)."""
    th0, ut, nu, dx, dt = _case(d, N, T, 71 + d)
    tt = th0 * 1.001
    m = O.Model(d, N, nu, dx, dt)
    for theta_target in (None, tt):
        ref = m.adjoint(th0, ut, T, theta_target=theta_target, checkpoint=0)
        for C in (1, 2, 3, 5, T):
            L, g, dnu = m.adjoint(th0, ut, T, theta_target=theta_target, checkpoint=C)
            assert L == ref[0] and np.array_equal(g, ref[1]) and dnu == ref[2], C


def test_oracle_results_do_not_depend_on_threads():
    """Node loops run on OpenMP threads; each node is computed as in a serial
    loop and sums over nodes are serial, so 1 and 4 threads agree bit for bit."""
    d, N, T = 2, (31, 20), 9
    th0, ut, nu, dx, dt = _case(d, N, T, 81)
    m = O.Model(d, N, nu, dx, dt)
    out = []
    before = O.threads()
    try:
        for n in (1, 4):
            O.set_threads(n)
            f0 = m.initialize(th0)
            f = m.run(f0, T)
            out.append((f0, f, m.recover(f), m.fd4_gradient(th0), m.adjoint(th0, ut, T, checkpoint=3)))
    finally:
        O.set_threads(before)
    a, b = out
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y)
    assert a[4][0] == b[4][0] and np.array_equal(a[4][1], b[4][1]) and a[4][2] == b[4][2]


def complex_forward_u(d, N, nu, dx, dt, th0, T):
    """u(T) of the forward map on a periodic grid, written out in complex
    arithmetic, for complex-step derivatives in nu (L(nu + ih), Im L / h).
    Independent of the oracle's code: the natural moments are the monomials
    of the (pinned) velocity list, 1; e_a; e_a^2; e_a e_b; e_a e_b^2 and
    e_a^2 e_b; e_a^2 e_b^2 (a < b), relaxed at 1, s1, s2x, s22, 1, 1
    (Sec. III.A); the relaxation set and weights are Eq. (Bur-Sol) and
    Eq. (d1-3-weight) in eps = nu dt / dx^2; f_0 = w theta0 - M^-1 S^-1 M g
    with g_k = w_k e_k . dx grad theta0 (FD4 gradient, Sec. IV); each step
    collides f* = f - M^-1 S M (f - w theta) and moves f*_i to x + e_i
    (Eq. (distribution-f)); u_a = (2 - s1) c sum_i e_ia f_i / theta
    (Eq. (ui-compute))."""
    e = O.lattice(d).astype(float)
    q = e.shape[0]
    eps = nu * dt / (dx * dx)
    a6 = 6.0 * eps + 1.0
    s1, s2x = 2.0 / a6, 24.0 * eps / (a6 * a6)
    if d == 1:
        s22, w1, wd = 1.0, 1.0 / 6.0, 0.0
    else:
        s22, w1, wd = 4.0 / (6.0 * eps + 3.0), 1.0 / 6.0 - (d - 1) * eps / 3.0, eps / 6.0
    nnz = np.count_nonzero(e, axis=1)
    w = np.where(nnz == 0, 1.0 - 2 * d * w1 - 2 * d * (d - 1) * wd, np.where(nnz == 1, w1, wd)).astype(complex)
    rows, rates = [np.ones(q)], [1.0]
    for a in range(d):
        rows.append(e[:, a])
        rates.append(s1)
    for a in range(d):
        rows.append(e[:, a] ** 2)
        rates.append(s2x)
    for a in range(d):
        for b in range(a + 1, d):
            rows += [e[:, a] * e[:, b], e[:, a] * e[:, b] ** 2, e[:, a] ** 2 * e[:, b], e[:, a] ** 2 * e[:, b] ** 2]
            rates += [s22, 1.0, 1.0, 1.0]
    M = np.array(rows)
    assert M.shape == (q, q)
    Minv = np.linalg.inv(M)
    S = np.array(rates, dtype=complex)
    coll = Minv @ (S[:, None] * M)
    init = Minv @ ((1.0 / S)[:, None] * M)
    ax = lambda a: d - 1 - a  # axis a (x first) is numpy axis d-1-a
    th0 = th0.astype(complex)
    grad = [(-np.roll(th0, -2, ax(a)) + 8 * np.roll(th0, -1, ax(a)) - 8 * np.roll(th0, 1, ax(a)) + np.roll(th0, 2, ax(a)))
            / (12.0 * dx) for a in range(d)]
    g = np.stack([w[k] * dx * sum(e[k, a] * grad[a] for a in range(d)) for k in range(q)])
    f = w.reshape((q,) + (1,) * d) * th0[None] - np.tensordot(init, g, axes=(1, 0))
    for _ in range(T):
        th = f.sum(axis=0)
        fs = f - np.tensordot(coll, f - w.reshape((q,) + (1,) * d) * th[None], axes=(1, 0))
        f = np.stack([np.roll(fs[i], tuple(int(e[i, a]) for a in range(d)), tuple(ax(a) for a in range(d)))
                      for i in range(q)])
    th = f.sum(axis=0)
    return np.stack([(2.0 - s1) * (dx / dt) * np.tensordot(e[:, a], f, axes=(0, 0)) / th for a in range(d)])


def _complex_step_loss(d, N, nu, dx, dt, th0, ut, T):
    """L = 1/2 sum (u(T) - ut)^2 from complex_forward_u."""
    return 0.5 * np.sum((complex_forward_u(d, N, nu, dx, dt, th0, T) - ut) ** 2)


@pytest.mark.parametrize("d,N,T", [(1, (12,), 9), (2, (6, 5), 6), (3, (4, 4, 3), 4)])
def test_oracle_dnu_matches_complex_step(d, N, T):
    """dL/dnu of the oracle's adjoint against the complex-step derivative of an
    independent complex-arithmetic forward map (no subtraction, so exact to
    rounding at h = 1e-20 nu): the real part reproduces the oracle's loss, the
    imaginary part its nu-gradient."""
    th0, ut, nu, dx, dt = _case(d, N, T, 71 + d)
    L, _, dnu = O.Model(d, N, nu, dx, dt).adjoint(th0, ut, T)
    h = 1e-20 * nu
    Lc = _complex_step_loss(d, N, nu + 1j * h, dx, dt, th0, ut, T)
    assert Lc.real == pytest.approx(L, rel=1e-13)
    assert Lc.imag / h == pytest.approx(dnu, rel=1e-12)
