"""Oracle pins: lattice, moment matrix, weights and the fourth-order relaxation set.

Each check compares the oracle against something the paper or mathematics
fixes independently of the oracle's own code: the printed velocity lists
(Eqs. (d1q3)-(d3q19)), the moment conditions (Eq. (conseved-moment)), the
fourth-order conditions R and Con (Eqs. (Con-1d), (Con-d),
(nabla-theta-con-d1), (nabla-theta-con-d2)) that Theorem 2 solves.
"""
import itertools

import numpy as np
import pytest

import oracle as O


def test_lattices_match_printed_lists(golden):
    rows = golden("paper_lattices.txt")
    for d in (1, 2, 3):
        e = O.lattice(d)
        assert e.shape == (1 + 2 * d * d, d)
        for r in rows:
            if int(r[0]) == d:
                axis = int(r[1])
                printed = np.array([int(v) for v in r[2:]])
                assert np.array_equal(e[:, axis], printed), (d, axis)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_general_lattice_is_the_DdQ_1_plus_2d2_set(d):
    # rest + 2d axis velocities + 2d(d-1) face diagonals, each exactly once
    e = O.lattice(d)
    want = {tuple([0] * d)}
    for a in range(d):
        for s in (1, -1):
            v = [0] * d
            v[a] = s
            want.add(tuple(v))
    for a, b in itertools.combinations(range(d), 2):
        for sa, sb in itertools.product((1, -1), repeat=2):
            v = [0] * d
            v[a], v[b] = sa, sb
            want.add(tuple(v))
    got = [tuple(int(x) for x in row) for row in e]
    assert len(got) == len(set(got)) == 1 + 2 * d * d
    assert set(got) == want


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_moment_matrix_rows_are_natural_moments(d):
    M, kind = O.moment_matrix(d)
    e = O.lattice(d).astype(float)
    q = 1 + 2 * d * d
    assert M.shape == (q, q)
    # the row families of Eqs. (d1q3)-(ddqq), built here from the velocities
    rows = [np.ones(q)] + [e[:, a] for a in range(d)] + [e[:, a] ** 2 for a in range(d)]
    pairs = list(itertools.combinations(range(d), 2))
    rows += [e[:, a] * e[:, b] for a, b in pairs]
    rows += [e[:, a] * e[:, b] ** 2 for a, b in pairs]
    rows += [e[:, a] ** 2 * e[:, b] for a, b in pairs]
    rows += [e[:, a] ** 2 * e[:, b] ** 2 for a, b in pairs]
    assert np.array_equal(M, np.array(rows))
    assert np.linalg.matrix_rank(M) == q
    assert list(kind) == [0] + [1] * d + [2] * d + [3] * len(pairs) + [4] * 2 * len(pairs) + [5] * len(pairs)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_model_inverse_and_collision_operators(d):
    m = O.Model(d, [3] * d, 0.01, 0.1, 0.1 * 0.1 * 10)
    mats = m.matrices()
    q = m.q
    assert np.allclose(mats["M"] @ mats["Minv"], np.eye(q), atol=1e-13)
    # S diag per family: Eqs. (d1q3)-(ddqq)
    _, kind = O.moment_matrix(d)
    p = m.params
    want = {0: p["s0"], 1: p["s1"], 2: p["s2x"], 3: p["s22"], 4: 1.0, 5: 1.0}
    assert np.allclose(mats["S"], [want[k] for k in kind])
    # Ccol is M^-1 S M and Cinv its inverse
    assert np.allclose(mats["C"] @ mats["Cinv"], np.eye(q), atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("eps", [0.02, 0.1, 0.2048])
def test_weights_moment_conditions(d, eps):
    """Eq. (conseved-moment): sum w = 1, sum w e = 0, sum w e e = (c_s/c)^2 I with
    c_s^2 = [2 w_1 + 4(d-1) w_{1+2d}] c^2."""
    p = O.paper_set(d, eps)
    w = O.weights(d, p["w1"], p["wd"])
    e = O.lattice(d).astype(float)
    sigma = 2 * p["w1"] + 4 * (d - 1) * p["wd"]
    assert abs(w.sum() - 1.0) < 4e-15
    assert np.allclose(w @ e, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), sigma * np.eye(d), atol=1e-15)
    # paper: c_s^2 = c^2/3 for every d at Eq. (Bur-Sol)
    assert abs(sigma - 1.0 / 3.0) < 1e-15


def _fourth_order_conditions(d, p):
    s1, s2, s22, w1, wd = p["s1"], p["s2x"], p["s22"], p["w1"], p["wd"]
    if d == 1:
        R1 = 6 * (s2 * (s1 - 1) + s1 ** 2 + s2 - 2 * s1) - s2 * s1 ** 2 \
            + 6 * w1 * (2 * s1 * (2 - s1) + s2 * (4 + s1 ** 2 - 6 * s1))
        C1 = 3 * s1 * (s2 + s1 - 2) - s1 ** 2 * s2 + 6 * w1 * (2 - s1) * (s1 + s2 * (1 - s1))
        return [R1, C1]
    W = w1 + 2 * (d - 1) * wd
    Rd1 = 6 * (s2 * (s1 - 1) + s1 ** 2 + s2 - 2 * s1) - s2 * s1 ** 2 \
        + 6 * W * (2 * s1 * (2 - s1) + s2 * (4 + s1 ** 2 - 6 * s1))
    Rd2 = (s1 ** 2 * wd * (2 * (s1 - 2) * (2 * s2 + s22) + s2 * s22 * (8 - 3 * s1))
           - 8 * s1 * s2 * s22 * W ** 2
           + s22 * (w1 ** 2 + 4 * (d - 1) * wd * (w1 + (d - 1) * wd))
           * (8 * (s1 + s2 - s1 ** 2 + (s1 - 1) * s1 * s2) + (2 - s2) * s1 ** 3))
    Cd1 = 3 * s1 * (s2 + s1 - 2) - s1 ** 2 * s2 + 6 * W * (2 - s1) * (s1 + s2 * (1 - s1))
    Cd2 = -(s22 * w1 ** 2 + 4 * s22 * (w1 + (d - 1) * wd) * wd * (d - 1)) * (s1 - 2) * (s1 + s2 - s1 * s2) \
        - s1 ** 2 * wd * (2 * s2 + s22 - 2 * s2 * s22)
    return [Rd1, Rd2, Cd1, Cd2]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("eps", [0.01, 0.05, 0.1, 0.16, 0.2048, 0.3, 0.45])
def test_paper_set_solves_theorem_2(d, eps):
    """Eq. (Bur-Sol) must satisfy every condition of Eq. (Bur-Con)."""
    p = O.paper_set(d, eps)
    xi = 1.0 / p["s1"] - 0.5
    assert abs((2 * p["w1"] + 4 * (d - 1) * p["wd"]) * xi - eps) < 1e-15
    for c in _fourth_order_conditions(d, p):
        assert abs(c) < 1e-14
    for s in (p["s1"], p["s2x"]) + ((p["s22"],) if d > 1 else ()):
        assert 0.0 < s < 2.0


def test_wrong_relaxation_set_violates_conditions():
    # a dropped term (s21 of the SRT-like choice s21 = s1) must be detected
    p = dict(O.paper_set(2, 0.2))
    p["s2x"] = p["s1"]
    assert max(abs(c) for c in _fourth_order_conditions(2, p)) > 1e-3


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fd4_gradient_is_fourth_order(d):
    errs = []
    for N in (16, 32):
        m = O.Model(d, [N] * d, 0.01, 1.0 / N, 1.0 / N ** 2)
        X = np.meshgrid(*[np.arange(N) / N] * d, indexing="ij")
        X = X[::-1]  # axis a of space is numpy axis d-1-a
        th = 2 + np.prod([np.sin(2 * np.pi * (a + 1) * X[a]) for a in range(d)], axis=0)
        g = m.fd4_gradient(th)
        ex = np.stack([2 * np.pi * (a + 1) * np.cos(2 * np.pi * (a + 1) * X[a])
                       * np.prod([np.sin(2 * np.pi * (b + 1) * X[b]) for b in range(d) if b != a], axis=0)
                       for a in range(d)])
        errs.append(np.max(np.abs(g - ex)))
    assert 3.7 < np.log2(errs[0] / errs[1]) < 4.3
