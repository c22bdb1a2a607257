"""Thin ctypes binding of the C ABI in include/lb.h (argument marshalling only).

The functions ``lb_create``, ``lb_set_theta0``, ``lb_step``, ``lb_macros``,
``lb_sum_theta``, ``lb_reduce``, ... keep the C names and signatures but take
torch tensors for device arrays; :class:`Solver` wraps one context.  Every
step of the method runs in the library's CUDA kernels; there is no Python or
CPU fallback: if the compiled library is missing or no GPU is present, the
calls raise.

Array conventions (as in the C ABI): scalar fields are contiguous float64
CUDA tensors of shape (N[d-1], ..., N[0]) (x fastest); vector fields have a
leading axis of length d, entry a being the component along axis a.
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ESTATE, LB_ETIMEOUT, LB_ENONPOS = range(7)
LB_FP64, LB_FP32_SHIFTED, LB_FX64 = 0, 1, 2
LB_PERIODIC, LB_MIRROR = 0, 1
_STATUS = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_ESTATE",
           5: "LB_ETIMEOUT", 6: "LB_ENONPOS"}

_lock = threading.Lock()
_lib = None


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class lb_relax(ctypes.Structure):
    _fields_ = [("paper_set", ctypes.c_int), ("s1", ctypes.c_double), ("s2x", ctypes.c_double),
                ("s22", ctypes.c_double), ("w1", ctypes.c_double), ("wd", ctypes.c_double),
                ("theta_ref", ctypes.c_double)]


def library_path():
    return _build.LIB


def load():
    """Load the compiled library (building it if the toolkit is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB) or not _build.up_to_date():
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        p64 = ctypes.POINTER(ctypes.c_int64)
        pd = ctypes.POINTER(ctypes.c_double)
        sigs = {
            "lb_create": ([ctypes.c_int, p64, dbl, dbl, dbl, ctypes.POINTER(lb_relax), ctypes.c_int, vp,
                           ctypes.POINTER(vp)], ctypes.c_int),
            "lb_destroy": ([vp], ctypes.c_int),
            "lb_get_params": ([vp, pd], ctypes.c_int),
            "lb_set_theta0": ([vp, vp, vp], ctypes.c_int),
            "lb_set_boundary": ([vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "lb_get_boundary": ([vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "lb_step": ([vp, i64], ctypes.c_int),
            "lb_get_step": ([vp, p64], ctypes.c_int),
            "lb_macros": ([vp, vp, vp, vp], ctypes.c_int),
            "lb_check": ([vp], ctypes.c_int),
            "lb_set_viscosity": ([vp, dbl], ctypes.c_int),
            "lb_set_blocking": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "lb_get_blocking": ([vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "lb_autotune": ([vp, ctypes.c_int, pd], ctypes.c_int),
            "lb_sum_theta": ([vp, pd], ctypes.c_int),
            "lb_reduce": ([vp, vp, vp, vp, vp, pd], ctypes.c_int),
            "lb_state_layout": ([vp, p64, p64, p64], ctypes.c_int),
            "lb_save_state": ([vp, vp], ctypes.c_int),
            "lb_load_state": ([vp, vp, i64], ctypes.c_int),
            "lb_last_error": ([vp], ctypes.c_char_p),
            "lb_reduce_static": ([ctypes.c_int, i64, vp, vp, vp, vp, vp, vp], ctypes.c_int),
            "lb_selftest_staging_timeout": ([dbl, vp, pd], ctypes.c_int),
            "lb_selftest_int_to_f64": ([vp, vp, i64, vp, vp, vp], ctypes.c_int),
            "lb_selftest_mulfx": ([vp, vp, i64, vp, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _ptr(t, what, dtype=torch.float64, numel=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous %s tensor" % (what, dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (what, numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _check(lib, ctx, status, call):
    if status != LB_OK:
        msg = lib.lb_last_error(ctx)
        raise LBError(status, "%s: %s" % (call, msg.decode() if msg else ""))


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------------------
# Same names as the C ABI.
# --------------------------------------------------------------------------

def lb_create(d, N, nu, dx, dt, relax=None, precision=LB_FP64, stream=None):
    lib = load()
    sizes = [int(n) for n in N]
    arr = (ctypes.c_int64 * max(3, len(sizes)))(*sizes)
    rs = lb_relax(1, 0, 0, 0, 0, 0, 0.0)
    if relax is not None:
        if relax.get("paper_set", False) or "s1" not in relax:
            rs.paper_set = 1
        else:
            rs.paper_set = 0
            rs.s1, rs.s2x, rs.s22 = relax["s1"], relax["s2x"], relax.get("s22", 1.0)
            rs.w1, rs.wd = relax["w1"], relax.get("wd", 0.0)
        rs.theta_ref = float(relax.get("theta_ref", 0.0))
    out = ctypes.c_void_p()
    st = lib.lb_create(int(d), arr, float(nu), float(dx), float(dt), ctypes.byref(rs), int(precision),
                       _stream_handle(stream), ctypes.byref(out))
    _check(lib, None, st, "lb_create")
    return out


def lb_destroy(ctx):
    load().lb_destroy(ctx)


def lb_get_params(ctx):
    lib = load()
    buf = (ctypes.c_double * 15)()
    _check(lib, ctx, lib.lb_get_params(ctx, buf), "lb_get_params")
    keys = ("eps", "c", "cs2", "s1", "s2x", "s22", "w0", "w1", "wd", "nu", "dx", "dt", "q", "theta_ref",
            "fx_bits")
    return dict(zip(keys, list(buf)))


def lb_set_boundary(ctx, kinds):
    """kinds: one LB_PERIODIC / LB_MIRROR (or "periodic" / "mirror") per axis."""
    lib = load()
    names = {"periodic": LB_PERIODIC, "mirror": LB_MIRROR}
    vals = [names[k] if isinstance(k, str) else int(k) for k in kinds]
    arr = (ctypes.c_int * max(1, len(vals)))(*vals)
    _check(lib, ctx, lib.lb_set_boundary(ctx, arr), "lb_set_boundary")


def lb_get_boundary(ctx, d):
    lib = load()
    arr = (ctypes.c_int * 4)()
    _check(lib, ctx, lib.lb_get_boundary(ctx, arr), "lb_get_boundary")
    return ["mirror" if arr[a] == LB_MIRROR else "periodic" for a in range(d)]


def lb_set_theta0(ctx, theta0, grad_theta0=None, nodes=None, d=None):
    lib = load()
    n = nodes
    st = lib.lb_set_theta0(ctx, _ptr(theta0, "theta0", numel=n),
                           _ptr(grad_theta0, "grad_theta0", numel=None if n is None else n * d))
    _check(lib, ctx, st, "lb_set_theta0")


def lb_step(ctx, nsteps):
    lib = load()
    _check(lib, ctx, lib.lb_step(ctx, int(nsteps)), "lb_step")


def lb_get_step(ctx):
    lib = load()
    v = ctypes.c_int64()
    _check(lib, ctx, lib.lb_get_step(ctx, ctypes.byref(v)), "lb_get_step")
    return v.value


def lb_macros(ctx, theta=None, grad_theta=None, u=None):
    lib = load()
    st = lib.lb_macros(ctx, _ptr(theta, "theta"), _ptr(grad_theta, "grad_theta"), _ptr(u, "u"))
    _check(lib, ctx, st, "lb_macros")


def lb_check(ctx):
    """Synchronise and raise LBError for any device-side flag set since the last report."""
    lib = load()
    _check(lib, ctx, lib.lb_check(ctx), "lb_check")


def lb_set_viscosity(ctx, nu):
    lib = load()
    _check(lib, ctx, lib.lb_set_viscosity(ctx, float(nu)), "lb_set_viscosity")


def lb_set_blocking(ctx, steps_per_launch, tile=64, threads=512):
    lib = load()
    _check(lib, ctx, lib.lb_set_blocking(ctx, int(steps_per_launch), int(tile), int(threads)), "lb_set_blocking")


def lb_get_blocking(ctx):
    lib = load()
    buf = (ctypes.c_int * 4)()
    _check(lib, ctx, lib.lb_get_blocking(ctx, buf), "lb_get_blocking")
    return {"steps_per_launch": buf[0], "tile": buf[1], "threads": buf[2], "tiles": buf[3]}


def lb_autotune(ctx, trial_steps=16):
    lib = load()
    buf = (ctypes.c_double * 4)()
    _check(lib, ctx, lib.lb_autotune(ctx, int(trial_steps), buf), "lb_autotune")
    return {"steps_per_launch": int(buf[0]), "tile": int(buf[1]), "threads": int(buf[2]), "us_per_step": buf[3]}


def lb_sum_theta(ctx):
    lib = load()
    v = ctypes.c_double()
    _check(lib, ctx, lib.lb_sum_theta(ctx, ctypes.byref(v)), "lb_sum_theta")
    return v.value


def lb_reduce(ctx, theta, u, exact_theta, exact_u, d):
    lib = load()
    buf = (ctypes.c_double * (3 * (d + 1) + 1))()
    st = lib.lb_reduce(ctx, _ptr(theta, "theta"), _ptr(u, "u"), _ptr(exact_theta, "exact_theta"),
                       _ptr(exact_u, "exact_u"), buf)
    _check(lib, ctx, st, "lb_reduce")
    vals = list(buf)
    names = ["theta"] + ["u%d" % a for a in range(d)]
    out = {nm: {"rmse": vals[3 * v], "linf": vals[3 * v + 1], "rel_l2": vals[3 * v + 2]}
           for v, nm in enumerate(names)}
    out["sum_theta"] = vals[-1]
    return out


def lb_reduce_static(d, nodes, theta, u, exact_theta, exact_u, out, stream=None):
    """Allocation-free error norms (device output ``out`` of 3(d+1)+1 doubles),
    for callers that cannot allocate device memory; see include/lb.h.  The
    tensors must hold exactly ``nodes`` (theta fields) and ``d * nodes``
    (velocity fields) values and lie on the current device."""
    lib = load()
    d, nodes = int(d), int(nodes)
    # sizes the library serves are checked against the tensors here; others
    # go to the library, which rejects them (LB_EINVAL)
    n = nodes if (1 <= d <= 3 and 1 <= nodes <= (1 << 31)) else None
    if n is not None:
        dev = torch.cuda.current_device()
        for name, t in (("theta", theta), ("u", u), ("exact_theta", exact_theta), ("exact_u", exact_u),
                        ("out", out)):
            if isinstance(t, torch.Tensor) and t.is_cuda and t.device.index != dev:
                raise ValueError("%s is on cuda:%d, not the current device cuda:%d" % (name, t.device.index, dev))
        if not isinstance(out, torch.Tensor) or out.numel() < 3 * (d + 1) + 1:
            raise ValueError("out must hold at least 3(d+1)+1 = %d doubles" % (3 * (d + 1) + 1))
    st = lib.lb_reduce_static(d, nodes, _ptr(theta, "theta", numel=n), _ptr(u, "u", numel=None if n is None else d * n),
                              _ptr(exact_theta, "exact_theta", numel=n),
                              _ptr(exact_u, "exact_u", numel=None if n is None else d * n),
                              _ptr(out, "out"), _stream_handle(stream))
    if st != LB_OK:
        raise LBError(st, "lb_reduce_static")


def lb_selftest_staging_timeout(limit_s=0.05, stream=None):
    """(status, seconds waited) of the bounded-wait self-test (LB_ETIMEOUT expected)."""
    lib = load()
    w = ctypes.c_double()
    st = lib.lb_selftest_staging_timeout(float(limit_s), _stream_handle(stream), ctypes.byref(w))
    return st, w.value


def lb_selftest_int_to_f64(hi, lo, stream=None):
    """(out128, out64): the library's integer -> FP64 conversions of the
    128-bit integers hi * 2^64 + lo and of lo read as int64 (CUDA int64
    tensors of equal length; lo holds the unsigned low words' bit patterns)."""
    lib = load()
    if not (isinstance(hi, torch.Tensor) and isinstance(lo, torch.Tensor) and hi.is_cuda and lo.is_cuda
            and hi.dtype == torch.int64 and lo.dtype == torch.int64 and hi.is_contiguous() and lo.is_contiguous()
            and hi.numel() == lo.numel()):
        raise TypeError("hi and lo must be contiguous CUDA int64 tensors of equal length")
    o128 = torch.empty(hi.numel(), dtype=torch.float64, device=hi.device)
    o64 = torch.empty(hi.numel(), dtype=torch.float64, device=hi.device)
    st = lib.lb_selftest_int_to_f64(ctypes.c_void_p(hi.data_ptr()), ctypes.c_void_p(lo.data_ptr()), hi.numel(),
                                    ctypes.c_void_p(o128.data_ptr()), ctypes.c_void_p(o64.data_ptr()),
                                    _stream_handle(stream))
    if st != LB_OK:
        raise LBError(st, "lb_selftest_int_to_f64")
    return o128, o64


def lb_selftest_mulfx(a, k, stream=None):
    """(split, wide): the fixed-point collision product round(a * k / 2^62)
    from the split-word form the collisions use and from a 128-bit product
    (contiguous CUDA int64 tensors of equal length)."""
    lib = load()
    if not (isinstance(a, torch.Tensor) and isinstance(k, torch.Tensor) and a.is_cuda and k.is_cuda
            and a.dtype == torch.int64 and k.dtype == torch.int64 and a.is_contiguous() and k.is_contiguous()
            and a.numel() == k.numel()):
        raise TypeError("a and k must be contiguous CUDA int64 tensors of equal length")
    split = torch.empty_like(a)
    wide = torch.empty_like(a)
    st = lib.lb_selftest_mulfx(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(k.data_ptr()), a.numel(),
                               ctypes.c_void_p(split.data_ptr()), ctypes.c_void_p(wide.data_ptr()),
                               _stream_handle(stream))
    if st != LB_OK:
        raise LBError(st, "lb_selftest_mulfx")
    return split, wide


def lb_state_layout(ctx):
    lib = load()
    p, s, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib, ctx, lib.lb_state_layout(ctx, ctypes.byref(p), ctypes.byref(s), ctypes.byref(e)),
           "lb_state_layout")
    return p.value, s.value, e.value


def lb_save_state(ctx, buf):
    lib = load()
    _check(lib, ctx, lib.lb_save_state(ctx, ctypes.c_void_p(buf.data_ptr())), "lb_save_state")


def lb_load_state(ctx, buf, step):
    lib = load()
    _check(lib, ctx, lib.lb_load_state(ctx, ctypes.c_void_p(buf.data_ptr()), int(step)), "lb_load_state")


# --------------------------------------------------------------------------
# Convenience wrapper.
# --------------------------------------------------------------------------

class Solver:
    """One MRT-LB solver context on the current CUDA device.

    ``relax`` = None uses Theorem 2's relaxation set; a dict with s1, s2x,
    s22, w1, wd overrides it.  ``precision`` is "fp64" or "fp32s" (FP32
    shifted storage around ``theta_ref``) or "fx64" (64-bit fixed-point
    storage with exact integer moment sums).  ``boundary`` gives each axis
    "periodic" (default) or "mirror" (walls on the first and last node,
    d theta/dn = 0, i.e. zero normal velocity).
    """

    def __init__(self, d, N, nu, dx, dt, relax=None, precision="fp64", theta_ref=0.0, stream=None,
                 boundary=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the MRT-LB solver needs a CUDA GPU; no CPU fallback exists")
        self.d = int(d)
        self.N = tuple(int(n) for n in N)
        if len(self.N) != self.d:
            raise ValueError("N must have d entries")
        self.shape = tuple(reversed(self.N))
        self.nodes = 1
        for n in self.N:
            self.nodes *= n
        self.precision = {"fp64": LB_FP64, "fp32s": LB_FP32_SHIFTED, "fx64": LB_FX64}[precision]
        rel = dict(relax or {})
        rel["theta_ref"] = float(theta_ref)
        self.stream = stream
        self._lib = load()
        self.ctx = lb_create(self.d, self.N, nu, dx, dt, rel, self.precision, stream)
        if boundary is not None:
            if len(boundary) != self.d:
                raise ValueError("boundary must have d entries")
            lb_set_boundary(self.ctx, boundary)
        self.boundary = lb_get_boundary(self.ctx, self.d)
        self.params = lb_get_params(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, comps=0):
        shape = self.shape if comps == 0 else (comps,) + self.shape
        return torch.empty(shape, dtype=torch.float64, device="cuda")

    def set_theta0(self, theta0, grad_theta0=None):
        lb_set_theta0(self.ctx, theta0, grad_theta0, self.nodes, self.d)

    def step(self, n):
        lb_step(self.ctx, n)

    @property
    def nsteps(self):
        return lb_get_step(self.ctx)

    def macros(self, theta=None, grad=None, u=None, want=("theta", "grad", "u")):
        theta = theta if theta is not None or "theta" not in want else self._field()
        grad = grad if grad is not None or "grad" not in want else self._field(self.d)
        u = u if u is not None or "u" not in want else self._field(self.d)
        lb_macros(self.ctx, theta, grad, u)
        return theta, grad, u

    def sum_theta(self):
        return lb_sum_theta(self.ctx)

    def check(self):
        lb_check(self.ctx)

    def set_blocking(self, steps_per_launch, tile=64, threads=512):
        lb_set_blocking(self.ctx, steps_per_launch, tile, threads)

    def blocking(self):
        return lb_get_blocking(self.ctx)

    def autotune(self, trial_steps=16):
        """Pick one sweep per launch or blocked sweeps by timing; overwrites the state."""
        return lb_autotune(self.ctx, trial_steps)

    def set_viscosity(self, nu):
        lb_set_viscosity(self.ctx, nu)
        self.params = lb_get_params(self.ctx)

    def reduce(self, theta, u, exact_theta, exact_u):
        return lb_reduce(self.ctx, theta, u, exact_theta, exact_u, self.d)

    def state_layout(self):
        return lb_state_layout(self.ctx)

    def save_state(self):
        pitch, slab, eb = self.state_layout()
        q = int(self.params["q"])
        buf = torch.empty(q * slab * eb, dtype=torch.uint8, device="cuda")
        lb_save_state(self.ctx, buf)
        return buf

    def load_state(self, buf, step):
        lb_load_state(self.ctx, buf, step)


# --------------------------------------------------------------------------
# Batched 2D instances (include/lb_batch.h).
# --------------------------------------------------------------------------

_batch_sigs = {
    "lb_batch_create": (["i", "p64", "pd", "pd", "pd", "relax", "i", "vp", "pvp"], "i"),
    "lb_batch_destroy": (["vp"], "i"),
    "lb_batch_set_theta_ref": (["vp", "pd"], "i"),
    "lb_batch_set_theta0": (["vp", "vp", "vp"], "i"),
    "lb_batch_step": (["vp", "i64"], "i"),
    "lb_batch_macros": (["vp", "vp", "vp"], "i"),
    "lb_batch_errors": (["vp", "vp", "vp", "vp", "vp", "pd"], "i"),
    "lb_batch_autotune": (["vp", "i", "pd"], "i"),
    "lb_batch_set_schedule": (["vp", "d", "i", "i"], "i"),
    "lb_batch_schedule": (["vp", "pd"], "i"),
    "lb_batch_set_blocking": (["vp", "i", "i", "i", "i"], "i"),
    "lb_batch_last_error": (["vp"], "s"),
}


def _load_batch():
    lib = load()
    if getattr(lib, "_batch_ready", False):
        return lib
    m = {"i": ctypes.c_int, "i64": ctypes.c_int64, "d": ctypes.c_double, "vp": ctypes.c_void_p,
         "p64": ctypes.POINTER(ctypes.c_int64), "pd": ctypes.POINTER(ctypes.c_double),
         "relax": ctypes.POINTER(lb_relax), "pvp": ctypes.POINTER(ctypes.c_void_p), "s": ctypes.c_char_p}
    for name, (args, res) in _batch_sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = [m[a] for a in args]
        fn.restype = m[res]
    lib._batch_ready = True
    return lib


class Batch:
    """Many independent 2D periodic instances (D2Q9), advanced together.

    ``sizes`` is a list of (N0, N1); ``nu``, ``dx``, ``dt`` are per-instance
    sequences; relaxation sets follow Theorem 2 per instance.  Fields are
    concatenated in instance order (see include/lb_batch.h).
    """

    def __init__(self, sizes, nu, dx, dt, precision="fp32s", theta_ref=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the batched solver needs a CUDA GPU; no CPU fallback exists")
        self._lib = _load_batch()
        self.count = len(sizes)
        self.sizes = [tuple(int(n) for n in s) for s in sizes]
        self.nodes = [s[0] * s[1] for s in self.sizes]
        self.node_off = [0]
        for n in self.nodes:
            self.node_off.append(self.node_off[-1] + n)
        flat = (ctypes.c_int64 * (2 * self.count))(*[v for s in self.sizes for v in s])
        arr = lambda v: (ctypes.c_double * self.count)(*[float(x) for x in v])
        self.precision = {"fp64": LB_FP64, "fp32s": LB_FP32_SHIFTED, "fx64": LB_FX64}[precision]
        out = ctypes.c_void_p()
        st = self._lib.lb_batch_create(self.count, flat, arr(nu), arr(dx), arr(dt), None, self.precision,
                                       _stream_handle(stream), ctypes.byref(out))
        if st != LB_OK:
            raise LBError(st, "lb_batch_create")
        self.h = out
        if theta_ref is not None:
            self._call("lb_batch_set_theta_ref", arr(theta_ref))

    def _call(self, name, *args):
        st = getattr(self._lib, name)(self.h, *args)
        if st != LB_OK:
            msg = self._lib.lb_batch_last_error(self.h)
            raise LBError(st, "%s: %s" % (name, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "h", None):
            self._lib.lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def total_nodes(self):
        return self.node_off[-1]

    def set_theta0(self, theta0, grad0=None):
        self._call("lb_batch_set_theta0", _ptr(theta0, "theta0", numel=self.total_nodes),
                   _ptr(grad0, "grad0", numel=2 * self.total_nodes))

    def step(self, n):
        self._call("lb_batch_step", int(n))

    def macros(self, theta=None, u=None):
        theta = theta if theta is not None else torch.empty(self.total_nodes, dtype=torch.float64, device="cuda")
        u = u if u is not None else torch.empty(2 * self.total_nodes, dtype=torch.float64, device="cuda")
        self._call("lb_batch_macros", _ptr(theta, "theta"), _ptr(u, "u"))
        return theta, u

    def errors(self, theta, u, exact_theta, exact_u):
        buf = (ctypes.c_double * (4 * self.count))()
        self._call("lb_batch_errors", _ptr(theta, "theta"), _ptr(u, "u"), _ptr(exact_theta, "exact_theta"),
                   _ptr(exact_u, "exact_u"), buf)
        import numpy as np
        return np.array(list(buf)).reshape(self.count, 4)

    def autotune(self, trial_steps=10):
        buf = (ctypes.c_double * 6)()
        self._call("lb_batch_autotune", int(trial_steps), buf)
        return {"budget_bytes": buf[0], "threads": int(buf[1]), "groups": int(buf[2]), "us_per_step": buf[3],
                "steps_per_launch": int(buf[4]), "tile": int(buf[5])}

    def set_schedule(self, budget_bytes, threads=256, use_graph=True):
        self._call("lb_batch_set_schedule", float(budget_bytes), int(threads), int(bool(use_graph)))

    def set_blocking(self, steps_per_launch, tile=40, threads=512, use_graph=True):
        self._call("lb_batch_set_blocking", int(steps_per_launch), int(tile), int(threads), int(bool(use_graph)))

    def schedule(self):
        buf = (ctypes.c_double * 7)()
        self._call("lb_batch_schedule", buf)
        return {"budget_bytes": buf[0], "threads": int(buf[1]), "groups": int(buf[2]), "nodes": int(buf[3]),
                "steps_per_launch": int(buf[4]), "tile": int(buf[5]), "tiles": int(buf[6])}

    def split(self, flat, comps=1):
        """Per-instance views (shape (comps, N1, N0) or (N1, N0)) of a concatenated field."""
        out = []
        for j, (n0, n1) in enumerate(self.sizes):
            a = flat[comps * self.node_off[j]: comps * self.node_off[j + 1]]
            out.append(a.reshape((comps, n1, n0)) if comps > 1 else a.reshape((n1, n0)))
        return out


# --------------------------------------------------------------------------
# Discrete adjoint (include/lb_adjoint.h).
# --------------------------------------------------------------------------

_adj_sigs = {
    "lb_adjoint_create": (["vp", "i64", "i64", "i", "pvp"], "i"),
    "lb_adjoint_destroy": (["vp"], "i"),
    "lb_adjoint_forward": (["vp", "vp", "vp", "vp"], "i"),
    "lb_adjoint_seed": (["vp", "vp", "vp"], "i"),
    "lb_adjoint_step": (["vp", "i64"], "i"),
    "lb_adjoint_result": (["vp", "vp", "pd"], "i"),
    "lb_adjoint_info": (["vp", "pd"], "i"),
}


def _load_adj():
    lib = load()
    if getattr(lib, "_adj_ready", False):
        return lib
    m = {"i": ctypes.c_int, "i64": ctypes.c_int64, "vp": ctypes.c_void_p, "pd": ctypes.POINTER(ctypes.c_double),
         "pvp": ctypes.POINTER(ctypes.c_void_p)}
    for name, (args, res) in _adj_sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = [m[a] for a in args]
        fn.restype = m[res]
    lib._adj_ready = True
    return lib


class Adjoint:
    """Adjoint workspace over a :class:`Solver` (FP64 or FX64): forward with
    checkpoints, seed with dL/du at T, reverse steps, gradients."""

    def __init__(self, solver, T, checkpoint=0, want_nu=True):
        self._lib = _load_adj()
        self.solver = solver
        self.T = int(T)
        out = ctypes.c_void_p()
        st = self._lib.lb_adjoint_create(solver.ctx, self.T, int(checkpoint), int(bool(want_nu)), ctypes.byref(out))
        _check(self._lib, solver.ctx, st, "lb_adjoint_create")
        self.h = out
        self.want_nu = bool(want_nu)

    def close(self):
        if getattr(self, "h", None):
            self._lib.lb_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        _check(self._lib, self.solver.ctx, getattr(self._lib, name)(self.h, *args), name)

    def forward(self, theta0, theta=None, u=None):
        s = self.solver
        u = u if u is not None else torch.empty((s.d,) + s.shape, dtype=torch.float64, device="cuda")
        self._call("lb_adjoint_forward", _ptr(theta0, "theta0", numel=s.nodes), _ptr(theta, "theta"), _ptr(u, "u"))
        return u

    def seed(self, dL_du=None, dL_dtheta=None):
        """Seed with dL/du(T) (d*nodes) and/or dL/dtheta(T) (nodes); either may be None."""
        self._call("lb_adjoint_seed", _ptr(dL_du, "dL_du", numel=self.solver.d * self.solver.nodes),
                   _ptr(dL_dtheta, "dL_dtheta", numel=self.solver.nodes))

    def step(self, n):
        self._call("lb_adjoint_step", int(n))

    def result(self):
        g = torch.empty(self.solver.shape, dtype=torch.float64, device="cuda")
        dnu = ctypes.c_double(float("nan"))
        self._call("lb_adjoint_result", _ptr(g, "dL_dtheta0"), ctypes.byref(dnu) if self.want_nu else None)
        return g, (dnu.value if self.want_nu else None)

    def info(self):
        buf = (ctypes.c_double * 5)()
        self._call("lb_adjoint_info", buf)
        return {"T": int(buf[0]), "checkpoint": int(buf[1]), "checkpoints": int(buf[2]), "done": int(buf[3]),
                "bytes": int(buf[4])}


# --------------------------------------------------------------------------
# One slab of a grid cut along its slowest axis (include/lb_slab.h).
# --------------------------------------------------------------------------

_slab_sigs = {
    "lb_slab_create": (["i", "p64", "i", "i", "d", "d", "d", "relax", "i", "vp", "pvp"], "i"),
    "lb_slab_destroy": (["vp"], "i"),
    "lb_slab_info": (["vp", "p64"], "i"),
    "lb_slab_ctx": (["vp"], "vp"),
    "lb_slab_set_theta0": (["vp", "vp", "vp", "d"], "i"),
    "lb_slab_pack": (["vp", "vp", "vp"], "i"),
    "lb_slab_unpack": (["vp", "vp", "vp"], "i"),
    "lb_slab_step": (["vp"], "i"),
    "lb_slab_macros": (["vp", "vp", "vp", "vp"], "i"),
    "lb_slab_sum_theta": (["vp", "pd"], "i"),
}


def _load_slab():
    lib = load()
    if getattr(lib, "_slab_ready", False):
        return lib
    m = {"i": ctypes.c_int, "d": ctypes.c_double, "vp": ctypes.c_void_p, "p64": ctypes.POINTER(ctypes.c_int64),
         "pd": ctypes.POINTER(ctypes.c_double), "relax": ctypes.POINTER(lb_relax), "pvp": ctypes.POINTER(ctypes.c_void_p)}
    for name, (args, res) in _slab_sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = [m[a] for a in args]
        fn.restype = m[res]
    lib._slab_ready = True
    return lib


class Slab:
    """Part ``part`` of ``nparts`` of the periodic grid ``N``, cut along its
    slowest axis; see include/lb_slab.h.  A step is ``pack`` -> move the two
    buffers to the neighbours -> ``unpack`` -> ``step``; ``SlabRunner`` in
    ``slab.py`` does the moving between processes."""

    def __init__(self, d, N, part, nparts, nu, dx, dt, precision="fx64", theta_ref=0.0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the slab solver needs a CUDA GPU; no CPU fallback exists")
        self._lib = _load_slab()
        self.d, self.N, self.part, self.nparts = int(d), tuple(int(n) for n in N), int(part), int(nparts)
        arr = (ctypes.c_int64 * 4)(*(list(self.N) + [1] * (4 - self.d)))
        rs = lb_relax(1, 0, 0, 0, 0, 0, float(theta_ref))
        self.precision = {"fp64": LB_FP64, "fp32s": LB_FP32_SHIFTED, "fx64": LB_FX64}[precision]
        out = ctypes.c_void_p()
        st = self._lib.lb_slab_create(self.d, arr, self.part, self.nparts, float(nu), float(dx), float(dt),
                                      ctypes.byref(rs), self.precision, _stream_handle(stream), ctypes.byref(out))
        if st != LB_OK:
            raise LBError(st, "lb_slab_create: %s" % (self._lib.lb_last_error(None) or b"").decode())
        self.h = out
        info = (ctypes.c_int64 * 6)()
        self._lib.lb_slab_info(self.h, info)
        self.z0, self.nz, self.halo_count, self.elem, self.crossing, self.layer_nodes = list(info)
        self.ctx = ctypes.c_void_p(self._lib.lb_slab_ctx(self.h))
        self.dtype = {8: torch.int64 if self.precision == LB_FX64 else torch.float64, 4: torch.float32}[self.elem]
        # owned layers (lowest first) of a scalar field: shape (nz, ..., N0)
        self.shape = (self.nz,) + tuple(reversed(self.N[:-1]))

    def _call(self, name, *args):
        _check(self._lib, self.ctx, getattr(self._lib, name)(self.h, *args), name)

    def close(self):
        if getattr(self, "h", None):
            self._lib.lb_slab_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def halo_buffers(self, n=2):
        """n device buffers of one pack's size, in the storage type."""
        return [torch.empty(self.halo_count, dtype=self.dtype, device="cuda") for _ in range(n)]

    def set_theta0(self, theta0_ext, grad_ext, max_abs_theta0):
        """theta0 / grad theta0 on the owned layers plus one layer on each side."""
        n = (self.nz + 2) * self.layer_nodes
        self._call("lb_slab_set_theta0", _ptr(theta0_ext, "theta0", numel=n), _ptr(grad_ext, "grad", numel=self.d * n),
                   float(max_abs_theta0))

    def pack(self, send_down, send_up):
        self._call("lb_slab_pack", _ptr(send_down, "send_down", self.dtype, self.halo_count),
                   _ptr(send_up, "send_up", self.dtype, self.halo_count))

    def unpack(self, recv_down, recv_up):
        self._call("lb_slab_unpack", _ptr(recv_down, "recv_down", self.dtype, self.halo_count),
                   _ptr(recv_up, "recv_up", self.dtype, self.halo_count))

    def step(self):
        self._call("lb_slab_step")

    def macros(self):
        """(theta, grad theta, u) on the owned layers."""
        th = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        g = torch.empty((self.d,) + self.shape, dtype=torch.float64, device="cuda")
        u = torch.empty_like(g)
        self._call("lb_slab_macros", _ptr(th, "theta"), _ptr(g, "grad"), _ptr(u, "u"))
        return th, g, u

    def sum_theta(self):
        v = ctypes.c_double()
        self._call("lb_slab_sum_theta", ctypes.byref(v))
        return v.value
