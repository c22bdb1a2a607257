"""Seeded synthetic inputs and closed-form solutions (no LB arithmetic here).

This module builds the initial fields theta0 (and their exact gradients)
that the solver and the oracle both start from, plus the exact Cole-Hopf
solutions they are measured against.  It imports only numpy and holds none
of the lattice Boltzmann method: no lattice, no moments, no relaxation.

Every problem is a positive solution of the transformed diffusion equation
d(theta)/dt = nu * lap(theta) (Eq. (eq-theta)); the Burgers velocity is the
Cole-Hopf map u = -2 nu grad(theta)/theta (Eq. (transf)).

Array conventions: a scalar field on sizes N = (N_0, ..., N_{d-1}) has shape
(N_{d-1}, ..., N_0) (x fastest); a vector field has a leading axis of length
d, entry a being the component along axis a.  Nodes: x_a = origin + j*dx.
"""

from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


def grid(N, dx, origin=0.0):
    """Coordinate arrays (one per axis, x first) broadcast to the field shape."""
    d = len(N)
    axes = [origin + dx * np.arange(n, dtype=np.float64) for n in N]
    # field shape is (N_{d-1}, ..., N_0): axis a of space is numpy axis d-1-a
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return [mesh[d - 1 - a] for a in range(d)]


def cole_hopf_u(nu, theta, grad):
    """u = -2 nu grad(theta) / theta (Eq. (transf))."""
    return -2.0 * nu * grad / theta[None]


# --------------------------------------------------------------------------
# Problems: theta(x, t) and grad theta(x, t) in closed form.
# --------------------------------------------------------------------------

@dataclass
class FourierProblem:
    """theta = offset + sum_m a_m exp(-4 pi^2 nu |k_m|^2 t) cos(2 pi k_m . x + phi_m).

    Each mode solves the diffusion equation exactly, so the sum does too;
    the problem is periodic on the unit cube when every k_m is an integer
    vector.
    """

    d: int
    nu: float
    offset: float
    k: np.ndarray          # (modes, d) integer wave vectors
    amp: np.ndarray        # (modes,)
    phase: np.ndarray      # (modes,)
    origin: float = 0.0
    period: float = 1.0

    def _modes(self, N, dx, t):
        X = grid(N, dx, self.origin)
        for m in range(len(self.amp)):
            kk = self.k[m]
            arg = self.phase[m] + sum(2.0 * math.pi * kk[a] * X[a] / self.period for a in range(self.d))
            k2 = float(np.sum((2.0 * math.pi * kk / self.period) ** 2))
            decay = self.amp[m] * math.exp(-self.nu * k2 * t)
            yield kk, arg, decay

    def theta(self, N, dx, t=0.0):
        out = np.full(tuple(reversed(N)), self.offset, dtype=np.float64)
        for _, arg, decay in self._modes(N, dx, t):
            out += decay * np.cos(arg)
        return out

    def grad(self, N, dx, t=0.0):
        out = np.zeros((self.d,) + tuple(reversed(N)), dtype=np.float64)
        for kk, arg, decay in self._modes(N, dx, t):
            s = np.sin(arg)
            for a in range(self.d):
                out[a] -= decay * (2.0 * math.pi * kk[a] / self.period) * s
        return out

    def u(self, N, dx, t=0.0):
        return cole_hopf_u(self.nu, self.theta(N, dx, t), self.grad(N, dx, t))

    @staticmethod
    def random(d, nu, n_modes, kmax, amp_std, offset, seed, min_theta=0.5):
        """Seeded random positive field: k uniform over the integer vectors
        0 < |k| <= kmax, amplitudes ~ N(0, amp_std^2), phases ~ U[0, 2 pi).
        Redraws with seed + 1000 until min theta0 >= min_theta."""
        cand = [v for v in itertools.product(range(-kmax, kmax + 1), repeat=d)
                if 0 < sum(c * c for c in v) <= kmax * kmax]
        cand = np.array(cand, dtype=np.int64)
        s = seed
        while True:
            rng = np.random.default_rng(s)
            idx = rng.integers(0, len(cand), size=n_modes)
            amp = rng.normal(0.0, amp_std, size=n_modes)
            ph = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
            p = FourierProblem(d, nu, offset, cand[idx], amp, ph)
            if offset - np.sum(np.abs(amp)) >= min_theta:
                return p
            s += 1000


@dataclass
class ProductSineProblem:
    """theta = (A + exp(-nu pi^2 |kappa|^2 t) prod_a sin(pi kappa_a x_a)) / B.

    Covers the paper's periodic examples: Example 2 (kappa = (2, 1), A = 2,
    B = 2 on [0, 2]^2), Example 3 (kappa = (2, 1, 4), A = 2, B = 2 on
    [0, 2]^3) and Example 4 (kappa = (1, 2, 3, 4), A = 2, B = 1 on [-1, 1]^4),
    and the unit-domain sine tests (kappa = 2 per axis, A = 2, B = 1).
    """

    d: int
    nu: float
    kappa: tuple
    A: float = 2.0
    B: float = 1.0
    origin: float = 0.0

    @property
    def rate(self):
        return self.nu * math.pi ** 2 * sum(k * k for k in self.kappa)

    def theta(self, N, dx, t=0.0):
        X = grid(N, dx, self.origin)
        prod = np.ones(tuple(reversed(N)))
        for a in range(self.d):
            prod = prod * np.sin(math.pi * self.kappa[a] * X[a])
        return (self.A + math.exp(-self.rate * t) * prod) / self.B

    def grad(self, N, dx, t=0.0):
        X = grid(N, dx, self.origin)
        S = [np.sin(math.pi * self.kappa[a] * X[a]) for a in range(self.d)]
        C = [math.pi * self.kappa[a] * np.cos(math.pi * self.kappa[a] * X[a]) for a in range(self.d)]
        out = np.zeros((self.d,) + tuple(reversed(N)))
        dec = math.exp(-self.rate * t) / self.B
        for a in range(self.d):
            term = np.ones(tuple(reversed(N)))
            for b in range(self.d):
                term = term * (C[b] if b == a else S[b])
            out[a] = dec * term
        return out

    def u(self, N, dx, t=0.0):
        return cole_hopf_u(self.nu, self.theta(N, dx, t), self.grad(N, dx, t))


@dataclass
class ProductWaveProblem:
    """theta = (A + exp(-nu pi^2 |kappa|^2 t) prod_a w_a(pi kappa_a x_a)) / B
    with w_a = cos or sin per axis ("cos" on an axis with walls at x = 0 and
    x = (N_a - 1) dx = L_a: d theta/dn = 0 there for integer kappa_a L_a)."""

    d: int
    nu: float
    kappa: tuple
    waves: tuple
    A: float = 2.0
    B: float = 1.0

    @property
    def rate(self):
        return self.nu * math.pi ** 2 * sum(k * k for k in self.kappa)

    def _parts(self, N, dx):
        X = grid(N, dx)
        W, dW = [], []
        for a in range(self.d):
            k = math.pi * self.kappa[a]
            if self.waves[a] == "cos":
                W.append(np.cos(k * X[a]))
                dW.append(-k * np.sin(k * X[a]))
            else:
                W.append(np.sin(k * X[a]))
                dW.append(k * np.cos(k * X[a]))
        return W, dW

    def theta(self, N, dx, t=0.0):
        W, _ = self._parts(N, dx)
        prod = np.ones(tuple(reversed(N)))
        for a in range(self.d):
            prod = prod * W[a]
        return (self.A + math.exp(-self.rate * t) * prod) / self.B

    def grad(self, N, dx, t=0.0):
        W, dW = self._parts(N, dx)
        out = np.zeros((self.d,) + tuple(reversed(N)))
        dec = math.exp(-self.rate * t) / self.B
        for a in range(self.d):
            term = np.ones(tuple(reversed(N)))
            for b in range(self.d):
                term = term * (dW[b] if b == a else W[b])
            out[a] = dec * term
        return out

    def u(self, N, dx, t=0.0):
        return cole_hopf_u(self.nu, self.theta(N, dx, t), self.grad(N, dx, t))


def bessel_i_all(z, nmax, quad=1024):
    """I_0(z) .. I_nmax(z) from I_n(z) = (1/pi) int_0^pi exp(z cos s) cos(n s) ds,
    by the trapezoid rule over the full period (exponentially accurate for
    this periodic analytic integrand once quad >> z + nmax)."""
    s = 2.0 * math.pi * np.arange(quad) / quad
    spec = np.fft.rfft(np.exp(z * np.cos(s)))
    return spec.real[: nmax + 1] / quad


@dataclass
class WallBesselProblem:
    """Example 1 (Sec. V): 1D, u(x, 0) = sin(pi x) on [0, 1] with u = 0 at
    x = 0 and x = 1.  Its Cole-Hopf transform is
    theta(x, t) = a_0 + 2 sum_{n >= 1} a_n exp(-n^2 pi^2 nu t) cos(n pi x),
    a_n = I_n(1/(2 pi nu)) (modified Bessel functions of the first kind), and
    theta(x, 0) = exp(cos(pi x)/(2 pi nu)).  Nodes x_j = j dx, j = 0..N-1,
    with (N - 1) dx = 1."""

    nu: float
    nmax: int = 96

    def _coef(self):
        return bessel_i_all(1.0 / (2.0 * math.pi * self.nu), self.nmax)

    def _x(self, N, dx):
        return dx * np.arange(N[0], dtype=np.float64)

    def theta(self, N, dx, t=0.0):
        x = self._x(N, dx)
        if t == 0.0:  # closed form (the series cancels heavily where theta is small)
            return np.exp(np.cos(math.pi * x) / (2.0 * math.pi * self.nu))
        a = self._coef()
        n = np.arange(1, self.nmax + 1)
        w = a[1:] * np.exp(-(n * math.pi) ** 2 * self.nu * t)
        return a[0] + 2.0 * (w @ np.cos(math.pi * np.outer(n, x)))

    def grad(self, N, dx, t=0.0):
        x = self._x(N, dx)
        if t == 0.0:
            th = np.exp(np.cos(math.pi * x) / (2.0 * math.pi * self.nu))
            return (-np.sin(math.pi * x) / (2.0 * self.nu) * th)[None, :]
        a = self._coef()
        n = np.arange(1, self.nmax + 1)
        w = a[1:] * np.exp(-(n * math.pi) ** 2 * self.nu * t) * n * math.pi
        return (-2.0 * (w @ np.sin(math.pi * np.outer(n, x))))[None, :]

    def u(self, N, dx, t=0.0):
        return cole_hopf_u(self.nu, self.theta(N, dx, t), self.grad(N, dx, t))


# --------------------------------------------------------------------------
# The standard workloads (sizes, eps, steps).  eps = nu*dt/dx^2 is fixed per
# family so that t_end is an integer number of steps at every N.
# --------------------------------------------------------------------------

@dataclass
class Case:
    name: str
    d: int
    N: tuple
    nu: float
    dx: float
    dt: float
    nsteps: int
    problem: object
    extra: dict = field(default_factory=dict)

    @property
    def eps(self):
        return self.nu * self.dt / (self.dx * self.dx)

    @property
    def t_end(self):
        return self.nsteps * self.dt

    @property
    def nodes(self):
        return int(np.prod(self.N))


def sine_1d(N, nsteps=None):
    """1D, nu = 0.05, theta0 = 2 + sin(2 pi x) on [0,1), eps = 0.16, t_end = 0.1."""
    nu, eps = 0.05, 0.16
    dx = 1.0 / N
    dt = eps * dx * dx / nu
    steps = int(round(0.1 / dt)) if nsteps is None else nsteps
    return Case("sine1d_N%d" % N, 1, (N,), nu, dx, dt, steps,
                ProductSineProblem(1, nu, (2,), 2.0, 1.0))


def sine_2d(N, nsteps=None):
    """2D, nu = 0.02, theta0 = 2 + sin(2 pi x) sin(2 pi y), eps = 0.2048, t_end = 0.05."""
    nu, eps = 0.02, 0.2048
    dx = 1.0 / N
    dt = eps * dx * dx / nu
    steps = int(round(0.05 / dt)) if nsteps is None else nsteps
    return Case("sine2d_N%d" % N, 2, (N, N), nu, dx, dt, steps,
                ProductSineProblem(2, nu, (2, 2), 2.0, 1.0))


def fourier_3d(N, nsteps=None, seed=2311):
    """3D, nu = 0.01, 1.5 + 8 seeded modes |k| <= 3, a ~ N(0, 0.05^2),
    eps = 0.0512, t_end = 0.02."""
    nu, eps = 0.01, 0.0512
    dx = 1.0 / N
    dt = eps * dx * dx / nu
    steps = int(round(0.02 / dt)) if nsteps is None else nsteps
    prob = FourierProblem.random(3, nu, 8, 3, 0.05, 1.5, seed)
    return Case("fourier3d_N%d" % N, 3, (N, N, N), nu, dx, dt, steps, prob)


def paper_example(d, eps, level=0):
    """The paper's periodic Examples 2 (d = 2) and 3 (d = 3) at refinement
    `level` (dx halves, dt quarters per level), t = 2 (Sec. IV)."""
    if d == 2:
        dx0, dt0, kappa = 1.0 / 20, 1.0 / 50, (2, 1)
    elif d == 3:
        dx0, dt0, kappa = 1.0 / 10, 1.0 / 25, (2, 1, 4)
    else:
        raise ValueError("d must be 2 or 3")
    dx = dx0 / 2 ** level
    dt = dt0 / 4 ** level
    nu = eps * dx * dx / dt
    n = int(round(2.0 / dx))
    steps = int(round(2.0 / dt))
    return Case("paper_ex%d_eps%g_l%d" % (d, eps, level), d, (n,) * d, nu, dx, dt, steps,
                ProductSineProblem(d, nu, kappa, 2.0, 2.0))


def wall_example1(eps, level=0):
    """The paper's Example 1 (1D, walls at x = 0 and x = 1, t = 2) at
    refinement `level`: dx = 1/40 / 2^level, dt = 1/100 / 4^level,
    nu = eps dx^2 / dt; N = 1/dx + 1 nodes (both wall nodes included)."""
    dx = 1.0 / 40 / 2 ** level
    dt = 1.0 / 100 / 4 ** level
    nu = eps * dx * dx / dt
    n = int(round(1.0 / dx)) + 1
    steps = int(round(2.0 / dt))
    return Case("wall_ex1_eps%g_l%d" % (eps, level), 1, (n,), nu, dx, dt, steps, WallBesselProblem(nu))


def batched_2d(count=512, seed=2312, nsteps=2000):
    """Batched 2D: N_j log-uniform in [32, 512], nu_j log-uniform in
    [0.005, 0.1], dt = 4 dx^2 (so eps_j = 4 nu_j), theta0 = 1.5 + 6 seeded
    modes (|k| <= 3, amplitudes N(0, 0.05^2))."""
    rng = np.random.default_rng(seed)
    Ns = np.rint(np.exp(rng.uniform(math.log(32), math.log(512), size=count))).astype(int)
    nus = np.exp(rng.uniform(math.log(0.005), math.log(0.1), size=count))
    cases = []
    for j in range(count):
        N = int(Ns[j])
        dx = 1.0 / N
        dt = 4.0 * dx * dx
        prob = FourierProblem.random(2, float(nus[j]), 6, 3, 0.05, 1.5, seed * 7919 + j)
        cases.append(Case("batch%d_N%d" % (j, N), 2, (N, N), float(nus[j]), dx, dt, nsteps, prob))
    return cases


def adjoint_2d(N=512, nsteps=2000, seed=2313):
    """Adjoint 2D: nu = 0.02, eps = 0.2048, theta0 = 1.5 + 6 seeded modes;
    the target velocity comes from the same modes with amplitudes perturbed
    by N(0, 0.01^2)."""
    nu, eps = 0.02, 0.2048
    dx = 1.0 / N
    dt = eps * dx * dx / nu
    prob = FourierProblem.random(2, nu, 6, 3, 0.05, 1.5, seed)
    rng = np.random.default_rng(seed + 1)
    tgt = FourierProblem(2, nu, prob.offset, prob.k.copy(),
                         prob.amp + rng.normal(0.0, 0.01, size=len(prob.amp)), prob.phase.copy())
    return Case("adjoint2d_N%d" % N, 2, (N, N), nu, dx, dt, nsteps, prob, {"target": tgt})
