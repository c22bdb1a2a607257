"""Fourier-symbol pins of the oracle's time stepping.

For a single periodic mode, one step maps the pre-collision amplitudes by
G(k) = diag(exp(-i k . e_j dx)) K with K = I - M^-1 S M (I - w 1^T) (pull
streaming of the collided values).  Checked here:
* the oracle's run equals G(k)^n applied to the mode content of its own
  initial state (FFT), to rounding: this fixes the streaming direction, the
  collide-then-stream order and the storage convention independently of the
  stepping code;
* rho(G) <= 1 (stability at the paper's relaxation set);
* the eigenvalue of G closest to 1 decays at ln(lambda)/dt = -nu |k|^2 +
  O(dx^4): the error ratio on halving dx (dt ~ dx^2) is ~16, the paper's
  fourth-order claim seen on the symbol itself.
"""
import numpy as np
import pytest

import oracle as O


def _K(m):
    mats = m.matrices()
    q = m.q
    w = mats["w"]
    return np.eye(q) - mats["C"] @ (np.eye(q) - np.outer(w, np.ones(q))), mats["e"]


def _G(K, e, k, dx):
    return np.diag(np.exp(-1j * (e @ np.asarray(k, dtype=float)) * dx)) @ K


@pytest.mark.parametrize("d,N", [(1, (16,)), (2, (12, 10)), (3, (8, 6, 4))])
def test_run_equals_symbol_power(d, N):
    nu, eps = 0.03, 0.17
    dx = 1.0 / max(N)
    dt = eps * dx * dx / nu
    m = O.Model(d, N, nu, dx, dt)
    K, e = _K(m)
    kint = [1, 2, 1][:d]
    L = [n * dx for n in N]
    k = [2 * np.pi * kint[a] / L[a] for a in range(d)]
    axes = [dx * np.arange(n) for n in N]
    X = np.meshgrid(*reversed(axes), indexing="ij")
    X = [X[d - 1 - a] for a in range(d)]
    phase = sum(k[a] * X[a] for a in range(d))
    th0 = 1.5 + 0.2 * np.cos(phase + 0.3)
    g0 = np.stack([-0.2 * k[a] * np.sin(phase + 0.3) for a in range(d)])
    f0 = m.initialize(th0, g0)
    n = 9
    fn = m.run(f0, n)
    fft_axes = tuple(range(1, d + 1))
    idx = (slice(None),) + tuple(kint[d - 1 - a] for a in range(d))
    F0 = np.fft.fftn(f0, axes=fft_axes)[idx]
    Fn = np.fft.fftn(fn, axes=fft_axes)[idx]
    pred = np.linalg.matrix_power(_G(K, e, k, dx), n) @ F0
    assert np.max(np.abs(Fn - pred)) <= 1e-13 * np.max(np.abs(F0)) * np.prod(N)
    # the mean is a fixed point of K's conserved part: only modes 0 and +-k are present
    spec = np.abs(np.fft.fftn(fn, axes=fft_axes))
    spec[(slice(None),) + (0,) * d] = 0
    spec[idx] = 0
    neg = (slice(None),) + tuple((-kint[d - 1 - a]) % N[d - 1 - a] for a in range(d))
    spec[neg] = 0
    assert spec.max() <= 1e-12 * np.max(np.abs(F0))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_symbol_stable_and_fourth_order(d):
    nu, eps = 0.02, 0.12
    errs = []
    kint = np.array([1, 1, 2][:d], dtype=float)
    for n in (16, 32, 64):
        dx = 1.0 / n
        dt = eps * dx * dx / nu
        m = O.Model(d, (4,) * d, nu, dx, dt)
        K, e = _K(m)
        k = 2 * np.pi * kint
        lam = np.linalg.eigvals(_G(K, e, k, dx))
        assert np.max(np.abs(lam)) <= 1.0 + 1e-12
        top = lam[np.argmin(np.abs(lam - 1.0))]
        errs.append(abs(np.log(top).real / dt + nu * float(k @ k)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 <= r1 <= 19.0 and 14.0 <= r2 <= 18.0, (errs, r1, r2)
