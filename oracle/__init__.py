"""FP64 CPU oracle for the Cole-Hopf fourth-order MRT-LB method (arXiv:2309.02825).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` are the only callers.  The
product path (``paper_2309_02825_gb300``) never imports this package, and
this package imports nothing from it: the two share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain C, IEEE double, no fast-math,
no FP contraction), compiled to ``oracle/_build/liborc.so`` by :func:`build`.
This module only marshals numpy arrays.

Conventions: a scalar field on a ``d``-dimensional periodic grid with sizes
``N = (N_0, ..., N_{d-1})`` (``N_0`` along x, the fastest axis) is a numpy
array of shape ``(N_{d-1}, ..., N_0)``; a vector field has a leading axis of
length ``d`` whose entry ``a`` is the component along axis ``a`` (x first).
Distributions are arrays of shape ``(q, N_{d-1}, ..., N_0)``.  Nodes sit at
``x_a = j*dx``, ``j = 0..N_a-1``.

Parity status (each function is pinned in ``tests/test_oracle_*.py``):
lattice, moment matrix, relaxation set, weights, initialisation, step,
recovery, totals and the wall (mirror) model are all pinned; none is
"parity unpinned".
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build/liborc.so``, with
    OpenMP over the node loops when the compiler has it (the results do not
    depend on it: see ``set_threads``)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    r = subprocess.run(["gcc", *_CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        vp = ctypes.c_void_p
        lib.orc_q.argtypes = [ctypes.c_int]
        lib.orc_q.restype = ctypes.c_int
        lib.orc_lattice.argtypes = [ctypes.c_int, ip]
        lib.orc_moment_matrix.argtypes = [ctypes.c_int, ip, dp, ip]
        lib.orc_invert.argtypes = [ctypes.c_int, dp, dp]
        lib.orc_invert.restype = ctypes.c_int
        lib.orc_paper_set.argtypes = [ctypes.c_int, ctypes.c_double] + [dp] * 5
        lib.orc_weights.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_create.argtypes = [ctypes.c_int, lp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, dp]
        lib.orc_create.restype = vp
        lib.orc_free.argtypes = [vp]
        lib.orc_get_params.argtypes = [vp, dp]
        lib.orc_get_matrices.argtypes = [vp, dp, dp, dp, dp, dp, dp, ip]
        lib.orc_fd4_gradient.argtypes = [vp, dp, dp]
        lib.orc_initialize.argtypes = [vp, dp, dp, dp]
        lib.orc_step.argtypes = [vp, dp, dp]
        lib.orc_run.argtypes = [vp, dp, ctypes.c_long]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_recover.argtypes = [vp, dp, dp, dp, dp]
        lib.orc_total.argtypes = [vp, dp]
        lib.orc_total.restype = ctypes.c_double
        lib.orc_adjoint.argtypes = [vp, dp, dp, dp, ctypes.c_long, ctypes.c_long, dp, dp]
        lib.orc_adjoint.restype = ctypes.c_double
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        lib.orc_loss.argtypes = [vp, dp, dp, ctypes.c_long]
        lib.orc_loss.restype = ctypes.c_double
        _lib = lib
        return lib


def set_threads(n: int) -> None:
    """Host threads for the oracle's node loops (OpenMP).  Each node is
    computed as in a serial loop and sums over nodes are taken serially in
    node order, so results are bit-identical for every thread count."""
    _load().orc_set_threads(int(n))


def threads() -> int:
    """Threads the oracle's node loops use (1 without OpenMP)."""
    return int(_load().orc_get_threads())


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Building blocks (Sec. III.A)
# --------------------------------------------------------------------------

def lattice(d: int) -> np.ndarray:
    """Velocities e_i = c_i/c of DdQ(1+2d^2), shape (q, d) (Eqs. (d1q3)-(ddqq))."""
    lib = _load()
    q = lib.orc_q(d)
    e = np.zeros(q * d, dtype=np.int32)
    lib.orc_lattice(d, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e.reshape(q, d)


def moment_matrix(d: int):
    """Natural-moment matrix M (lattice units) and the family of each row."""
    lib = _load()
    e = lattice(d).astype(np.int32).ravel()
    q = lib.orc_q(d)
    M = np.zeros(q * q)
    kind = np.zeros(q, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_moment_matrix(d, e.ctypes.data_as(ip), _dp(M), kind.ctypes.data_as(ip))
    return M.reshape(q, q), kind


def paper_set(d: int, eps: float) -> dict:
    """Relaxation parameters and weights of Theorem 2, Eq. (Bur-Sol)."""
    lib = _load()
    out = [ctypes.c_double() for _ in range(5)]
    lib.orc_paper_set(d, float(eps), *[ctypes.byref(o) for o in out])
    s1, s2x, s22, w1, wd = (o.value for o in out)
    return {"s1": s1, "s2x": s2x, "s22": s22, "w1": w1, "wd": wd}


def weights(d: int, w1: float, wd: float) -> np.ndarray:
    """Weight vector of Eq. (d1-3-weight)."""
    lib = _load()
    q = lib.orc_q(d)
    w = np.zeros(q)
    lib.orc_weights(d, float(w1), float(wd), _dp(w))
    return w


# --------------------------------------------------------------------------
# Model
# --------------------------------------------------------------------------

class Model:
    """One periodic DdQ(1+2d^2) MRT-LB model (oracle).

    ``relax`` = None uses Eq. (Bur-Sol) with eps = nu*dt/dx^2; otherwise a
    dict with keys s1, s2x, s22, w1, wd.
    """

    def __init__(self, d, N, nu, dx, dt, relax=None):
        self._lib = _load()
        self.d = int(d)
        N = [int(n) for n in (N if np.ndim(N) else [N] * self.d)]
        if len(N) != self.d:
            raise ValueError("N must have d entries")
        self.N = tuple(N)
        self.shape = tuple(reversed(self.N))
        arr = (ctypes.c_long * 4)(*(N + [1] * (4 - len(N))))
        if relax is None:
            rs, paper = None, 1
        else:
            vals = [relax["s1"], relax["s2x"], relax["s22"], relax["w1"], relax["wd"]]
            rs, paper = (ctypes.c_double * 5)(*vals), 0
        self._h = self._lib.orc_create(self.d, arr, float(nu), float(dx), float(dt), paper, rs)
        if not self._h:
            raise ValueError("invalid model parameters")
        p = np.zeros(12)
        self._lib.orc_get_params(self._h, _dp(p))
        self.params = {
            "eps": p[0], "c": p[1], "cs2": p[2], "s0": p[3], "s1": p[4], "s2x": p[5],
            "s22": p[6], "w0": p[7], "w1": p[8], "wd": p[9], "nu": float(nu),
            "dx": float(dx), "dt": float(dt),
        }
        self.q = int(p[10])
        self.nodes = int(p[11])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    def matrices(self) -> dict:
        q, d = self.q, self.d
        M, Minv, C, Ci = (np.zeros(q * q) for _ in range(4))
        s, w = np.zeros(q), np.zeros(q)
        e = np.zeros(q * d, dtype=np.int32)
        self._lib.orc_get_matrices(self._h, _dp(M), _dp(Minv), _dp(s), _dp(w), _dp(C), _dp(Ci),
                                   e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return {"M": M.reshape(q, q), "Minv": Minv.reshape(q, q), "S": s, "w": w,
                "C": C.reshape(q, q), "Cinv": Ci.reshape(q, q), "e": e.reshape(q, d)}

    def fd4_gradient(self, theta):
        theta = _f64(theta).reshape(self.shape)
        g = np.zeros((self.d,) + self.shape)
        self._lib.orc_fd4_gradient(self._h, _dp(theta), _dp(g))
        return g

    def initialize(self, theta0, grad0=None):
        """Pre-collision f(x, 0) from the first two terms of Eq. (f-feq-o5)."""
        theta0 = _f64(theta0).reshape(self.shape)
        g = None if grad0 is None else _f64(grad0).reshape((self.d,) + self.shape)
        f = np.zeros((self.q,) + self.shape)
        self._lib.orc_initialize(self._h, _dp(theta0), _dp(g), _dp(f))
        return f

    def step(self, f):
        """One step of Eq. (distribution-f); returns a new array."""
        f = _f64(f)
        out = np.zeros_like(f)
        self._lib.orc_step(self._h, _dp(f), _dp(out))
        return out

    def run(self, f, nsteps):
        """nsteps steps; returns a new array."""
        f = _f64(f).copy()
        if self._lib.orc_run(self._h, _dp(f), int(nsteps)) != 0:
            raise MemoryError("oracle run")
        return f

    def recover(self, f):
        """(theta, grad theta, u) from pre-collision f (Sec. III.C)."""
        f = _f64(f)
        th = np.zeros(self.shape)
        g = np.zeros((self.d,) + self.shape)
        u = np.zeros((self.d,) + self.shape)
        self._lib.orc_recover(self._h, _dp(f), _dp(th), _dp(g), _dp(u))
        return th, g, u

    def total(self, f) -> float:
        return float(self._lib.orc_total(self._h, _dp(_f64(f))))

    def loss(self, theta0, utarget, T) -> float:
        """L = 1/2 sum (u(T) - utarget)^2 with f_0 from theta0 and its FD4 gradient."""
        th = _f64(theta0).reshape(self.shape)
        ut = _f64(utarget).reshape((self.d,) + self.shape)
        return float(self._lib.orc_loss(self._h, _dp(th), _dp(ut), int(T)))

    def adjoint(self, theta0, utarget, T, theta_target=None, checkpoint=0):
        """(L, dL/dtheta0, dL/dnu) by the discrete adjoint (paper relaxation set)
        for L = 1/2 sum |u(T) - utarget|^2 [+ 1/2 sum (theta(T) - theta_target)^2].
        ``checkpoint`` = 0 keeps every forward state; C > 0 keeps every C-th
        and recomputes one segment at a time (same results, bit for bit)."""
        th = _f64(theta0).reshape(self.shape)
        ut = _f64(utarget).reshape((self.d,) + self.shape)
        tt = None if theta_target is None else _f64(theta_target).reshape(self.shape)
        g = np.zeros(self.shape)
        de = ctypes.c_double()
        L = self._lib.orc_adjoint(self._h, _dp(th), _dp(ut), _dp(tt), int(T), int(checkpoint), _dp(g),
                                  ctypes.byref(de))
        if not np.isfinite(L):
            raise MemoryError("oracle adjoint")
        p = self.params
        return float(L), g, de.value * p["dt"] / (p["dx"] * p["dx"])


# --------------------------------------------------------------------------
# Walls with zero normal velocity (Example 1 of Sec. V: u = 0 at both ends).
# Under u = -2 nu grad theta / theta this is d theta / dn = 0, whose
# solutions are the restrictions of periodic solutions that are even about
# each wall.  The oracle therefore defines the scheme on a grid with walls as
# the periodic scheme on the grid doubled by even reflection, restricted to
# the original nodes: walls sit on the first and last node of a mirror axis
# (N_a nodes span (N_a - 1) dx) and the doubled axis is periodic with
# 2 (N_a - 1) nodes.
# --------------------------------------------------------------------------

def even_extension(a, d, mirror, vector=False):
    """Extend a field from N_a to 2(N_a - 1) nodes on each mirror axis by
    value(2(N_a - 1) - k) = value(k).  For a vector field (leading axis of
    length d) the component along a reflected axis is odd: it changes sign
    in the reflection and is zero on the wall nodes themselves."""
    a = np.array(a, dtype=np.float64)
    lead = 1 if vector else 0
    for ax in range(d):
        if not mirror[ax]:
            continue
        k = lead + (d - 1 - ax)  # array axis of grid axis ax (x is last)
        n = a.shape[k]
        if vector:
            sl = [slice(None)] * a.ndim
            sl[0] = ax
            for j in (0, n - 1):
                sl[k] = j
                a[tuple(sl)] = 0.0
        refl = np.flip(np.take(a, np.arange(1, n - 1), axis=k), axis=k)
        if vector:
            refl = refl.copy()
            refl[ax] *= -1.0
        a = np.concatenate([a, refl], axis=k)
    return a


def restrict(a, d, N, vector=False):
    """The original N nodes of a field on the doubled grid."""
    lead = 1 if vector else 0
    idx = [slice(None)] * lead + [slice(0, n) for n in reversed(N)]
    return np.ascontiguousarray(np.asarray(a)[tuple(idx)])


class MirrorModel:
    """The scheme on a grid whose axes ``mirror[a]`` have walls (the others
    periodic): a periodic :class:`Model` on the doubled grid, with theta0 and
    grad theta0 extended evenly (grad oddly along the wall normal) and the
    recovered fields restricted.  Distributions live on the doubled grid."""

    def __init__(self, d, N, mirror, nu, dx, dt, relax=None):
        self.d = int(d)
        self.N = tuple(int(n) for n in N)
        self.mirror = tuple(bool(m) for m in mirror)
        if len(self.N) != self.d or len(self.mirror) != self.d:
            raise ValueError("N and mirror must have d entries")
        if any(m and n < 3 for m, n in zip(self.mirror, self.N)):
            raise ValueError("a mirror axis needs at least 3 nodes")
        full = tuple(2 * (n - 1) if m else n for n, m in zip(self.N, self.mirror))
        self.full = Model(self.d, full, nu, dx, dt, relax)
        self.params, self.q = self.full.params, self.full.q

    def initialize(self, theta0, grad0=None):
        th = even_extension(theta0, self.d, self.mirror)
        g = None if grad0 is None else even_extension(grad0, self.d, self.mirror, vector=True)
        return self.full.initialize(th, g)

    def run(self, f, nsteps):
        return self.full.run(f, nsteps)

    def recover(self, f):
        th, g, u = self.full.recover(f)
        return (restrict(th, self.d, self.N), restrict(g, self.d, self.N, True),
                restrict(u, self.d, self.N, True))

    def wall_weights(self):
        """1/2 per wall a node lies on: the doubled grid holds every interior
        node 2^k times (k mirror axes) and a wall node half as often."""
        w = np.ones(tuple(reversed(self.N)))
        for ax in range(self.d):
            if self.mirror[ax]:
                k = self.d - 1 - ax
                sl = [slice(None)] * self.d
                for j in (0, self.N[ax] - 1):
                    sl[k] = j
                    w[tuple(sl)] *= 0.5
        return w

    def total(self, f) -> float:
        """Wall-weighted sum of theta = (sum over the doubled grid) / 2^k."""
        return self.full.total(f) / 2.0 ** sum(self.mirror)


# --------------------------------------------------------------------------
# Error metrics (Sec. IV): RMSE per variable, max error, convergence rate.
# --------------------------------------------------------------------------

def rmse(num, exact) -> float:
    """sqrt(mean over all nodes of (psi - psi*)^2), one variable at a time."""
    diff = np.asarray(num, dtype=np.float64) - np.asarray(exact, dtype=np.float64)
    return float(np.sqrt(np.mean(diff * diff)))


def linf(num, exact) -> float:
    return float(np.max(np.abs(np.asarray(num, dtype=np.float64) - np.asarray(exact, dtype=np.float64))))


def convergence_rate(err_coarse, err_fine, h_coarse, h_fine) -> float:
    """log(E_1/E_2)/log(h_1/h_2); equals the paper's CR for h_1/h_2 = 2."""
    return float(np.log(err_coarse / err_fine) / np.log(h_coarse / h_fine))
