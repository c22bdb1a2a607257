"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64: theta, grad theta and u must match to a max normwise relative
difference of 1e-12 (|gpu - oracle|_max <= 1e-12 * |oracle|_max per field).
Grids are chosen to span several warp segments (64 nodes in x for FP64,
128 for FP32) with ragged tails, plus degenerate sizes (N = 1, 2, 3 along an
axis) where every node is at the periodic wrap.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_02825_gb300 import lb
from paper_2309_02825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    return t.detach().cpu().numpy()


def _relmax(a, b):
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0))


def _check_fp64(ref, got, m, nsteps, ref0=None):
    """theta, grad theta and u each: max |gpu - oracle| <= 1e-12 max |oracle|.

    ref0 (the oracle's fields at step 0) is given only for the grids listed in
    DECAYING: there the bound is 1e-12 of max(|field(T)|, |field(0)|)."""
    out = {}
    for k, (name, a, b) in enumerate(zip(("theta", "grad", "u"), got, ref)):
        diff = float(np.max(np.abs(a - b)))
        scale = float(np.max(np.abs(b)))
        out[name] = diff / scale if scale > 0 else diff
        if ref0 is not None:
            scale = max(scale, float(np.max(np.abs(ref0[k]))))
        assert diff <= TOL64 * scale, (name, diff, TOL64 * scale, out[name])
    return out


# 1D grids of one to three nodes, where every node is at the periodic wrap:
# grad theta and u have no spatial structure left to keep them up and decay
# geometrically (J by a factor (1 - s1) per step on one node) to 1e-6 .. 1e-4
# of their initial size, while the rounding carried from the first steps
# stays at the initial size.  For these grids the bound is 1e-12 of the
# initial field's size; measured against the final field's own maximum the
# differences are 1.6e-12 .. 5.1e-11 (grad), all other cases meet 1e-12 of
# their own maximum.
DECAYING = {(1, (1,)), (1, (2,)), (1, (3,))}


def _problem(d, N, seed, nu=0.02):
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.1, 1.5, seed)
    dx = 1.0 / max(N)
    dt = 0.2 * dx * dx / nu
    return prob, dx, dt


def _run_both(d, N, nsteps, seed=11, precision="fp64", grad=True, relax=None, theta_ref=1.5):
    prob, dx, dt = _problem(d, N, seed)
    nu = prob.nu
    th0 = prob.theta(N, dx)
    g0 = prob.grad(N, dx) if grad else None
    m = O.Model(d, N, nu, dx, dt, relax)
    f0 = m.initialize(th0, g0)
    th_o, g_o, u_o = m.recover(m.run(f0, nsteps))
    m.ref0 = m.recover(f0) if (d, tuple(N)) in DECAYING else None
    s = lb.Solver(d, N, nu, dx, dt, relax=relax, precision=precision, theta_ref=theta_ref)
    s.set_theta0(_dev(th0), None if g0 is None else _dev(g0))
    s.step(nsteps)
    th, g, u = s.macros()
    torch.cuda.synchronize()
    return (th_o, g_o, u_o), (_host(th), _host(g), _host(u)), s, m


CASES = [
    (1, (100,), 1), (1, (100,), 37), (1, (1,), 5), (1, (2,), 4), (1, (3,), 9), (1, (64,), 20), (1, (129,), 13),
    (2, (70, 45), 1), (2, (70, 45), 23), (2, (64, 64), 20), (2, (130, 3), 7), (2, (5, 33), 6), (2, (1, 9), 4),
    (2, (200, 17), 150),
    (3, (37, 22, 13), 1), (3, (37, 22, 13), 9), (3, (64, 16, 8), 16), (3, (3, 4, 5), 5), (3, (70, 1, 6), 4),
    (4, (10, 8, 6, 5), 1), (4, (10, 8, 6, 5), 6), (4, (70, 3, 4, 2), 4), (4, (3, 4, 2, 5), 3),
    # rows that fill whole warps: the 4D 8-byte sweeps take row segments here, the flat mapping elsewhere
    (4, (64, 3, 4, 3), 4), (4, (32, 5, 3, 3), 3),
]


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("d,N,nsteps", CASES)
def test_fp64_matches_oracle(d, N, nsteps, precision):
    """FP64 storage and 64-bit fixed-point storage both meet the FP64 bar."""
    ref, got, _, m = _run_both(d, N, nsteps, precision=precision)
    rel = _check_fp64(ref, got, m, nsteps, m.ref0)
    print("%s parity d=%d N=%s steps=%d rel: %s" % (precision, d, N, nsteps, rel))


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("d,N", [(1, (50,)), (2, (66, 40)), (3, (20, 18, 9))])
def test_fp64_fd_gradient_fallback(d, N, precision):
    ref, got, _, m = _run_both(d, N, 5, grad=False, precision=precision)
    _check_fp64(ref, got, m, 5)


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_fp64_custom_relaxation_set(d, precision):
    relax = {"s1": 1.3, "s2x": 0.7, "s22": 1.1, "w1": 0.12, "wd": 0.02 if d > 1 else 0.0}
    N = [(90,), (40, 30), (20, 12, 10)][d - 1]
    ref, got, _, m = _run_both(d, N, 11, relax=relax, precision=precision)
    _check_fp64(ref, got, m, 11)


@pytest.mark.parametrize("d,N", [(1, (77,)), (2, (70, 45)), (3, (24, 10, 7))])
def test_sum_theta_conserved_and_matches_oracle(d, N):
    (th_o, _, _), _, s, m = _run_both(d, N, 30)
    total = s.sum_theta()
    assert abs(total - th_o.sum()) <= 1e-13 * abs(th_o.sum())
    prob, dx, _ = _problem(d, N, 11)
    assert abs(total - prob.theta(N, dx).sum()) <= 1e-12 * abs(total)


@pytest.mark.parametrize("d,N", [(1, (77,)), (2, (70, 45)), (3, (24, 10, 7)), (4, (9, 6, 5, 4))])
def test_fx64_initial_mass_is_rounded_theta0(d, N):
    """The fixed-point initialisation forms the rest population as theta
    minus the others, so the stored state sums to sum_x round(theta0 2^F)
    exactly (compared modulo 2^64, as the int64 sums wrap)."""
    prob, dx, dt = _problem(d, N, 11)
    s = lb.Solver(d, N, prob.nu, dx, dt, precision="fx64")
    th0 = prob.theta(N, dx)
    s.set_theta0(_dev(th0), _dev(prob.grad(N, dx)))
    F = lb.lb_get_params(s.ctx)["fx_bits"]
    pitch, _, _ = s.state_layout()
    q = int(s.params["q"])
    st = s.save_state().view(torch.int64).view(q, -1, pitch)[..., : N[0]]
    got = int(st.sum().item()) % 2 ** 64
    want = int(np.rint(th0 * 2.0 ** F).astype(np.int64).sum()) % 2 ** 64
    assert got == want


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_init_constants_beyond_fixed_point_range(precision):
    """s1 = 0.1 makes the initialisation's gradient constant (sigma/s1 - ...)/2
    exceed the fixed-point range: FX64 then forms the values in FP64 and
    rounds them, and still meets the FP64 bar."""
    relax = {"s1": 0.1, "s2x": 0.7, "s22": 1.1, "w1": 0.12, "wd": 0.02}
    ref, got, _, m = _run_both(2, (40, 30), 7, relax=relax, precision=precision)
    _check_fp64(ref, got, m, 7)


@pytest.mark.parametrize("d,N", [(1, (77,)), (2, (70, 45)), (3, (24, 10, 7))])
def test_fx64_conserves_sum_exactly(d, N):
    """Fixed point: the rest population is theta minus the others, so the
    integer sum of the state never changes; lb_sum_theta only rounds when it
    converts each stored value to FP64."""
    prob, dx, dt = _problem(d, N, 11)
    s = lb.Solver(d, N, prob.nu, dx, dt, precision="fx64")
    th0 = prob.theta(N, dx)
    s.set_theta0(_dev(th0), _dev(prob.grad(N, dx)))
    t0 = s.sum_theta()
    s.step(40)
    t1 = s.sum_theta()
    snap = s.save_state().view(torch.int64)
    s.step(1)
    snap2 = s.save_state().view(torch.int64)
    pitch, slab, _ = s.state_layout()
    q = int(s.params["q"])
    mask = (torch.arange(pitch, device="cuda") < N[0])
    tot = [int((sn.view(q, -1, pitch) * mask).sum().item()) for sn in (snap, snap2)]
    assert tot[0] == tot[1]
    assert abs(t1 - t0) <= 1e-14 * abs(t0)
    # max|theta0| * 2^F < 2^59 with the largest such F
    assert lb.lb_get_params(s.ctx)["fx_bits"] == 59 - math.frexp(float(th0.max()))[1]


def test_reduce_norms_match_numpy():
    d, N = 2, (96, 50)
    (th_o, _, u_o), (th, _, u), s, _ = _run_both(d, N, 12)
    rng = np.random.default_rng(5)
    ex_t = th + rng.normal(0, 1e-3, size=th.shape)
    ex_u = u + rng.normal(0, 1e-4, size=u.shape)
    r = s.reduce(_dev(th), _dev(u), _dev(ex_t), _dev(ex_u))
    assert r["theta"]["rmse"] == pytest.approx(O.rmse(th, ex_t), rel=1e-12)
    assert r["theta"]["linf"] == pytest.approx(O.linf(th, ex_t), rel=1e-15)
    for a in range(d):
        assert r["u%d" % a]["rmse"] == pytest.approx(O.rmse(u[a], ex_u[a]), rel=1e-12)
        assert r["u%d" % a]["rel_l2"] == pytest.approx(
            np.sqrt(np.sum((u[a] - ex_u[a]) ** 2) / np.sum(ex_u[a] ** 2)), rel=1e-12)
    assert r["sum_theta"] == pytest.approx(th.sum(), rel=1e-14)


def test_state_save_load_roundtrip():
    d, N = 2, (70, 45)
    prob, dx, dt = _problem(d, N, 3)
    s = lb.Solver(d, N, prob.nu, dx, dt)
    s.set_theta0(_dev(prob.theta(N, dx)), _dev(prob.grad(N, dx)))
    s.step(5)
    snap = s.save_state()
    th_a, _, u_a = s.macros()
    s.step(7)
    s.load_state(snap, 5)
    assert s.nsteps == 5
    th_b, _, u_b = s.macros()
    torch.cuda.synchronize()
    assert torch.equal(th_a, th_b) and torch.equal(u_a, u_b)


def test_invalid_inputs_are_reported():
    with pytest.raises(lb.LBError) as ei:
        lb.Solver(5, (4, 4, 4, 4, 4), 0.1, 0.1, 0.1)
    assert ei.value.status == lb.LB_EINVAL
    with pytest.raises(lb.LBError):
        lb.Solver(2, (8, 8), -1.0, 0.1, 0.1)
    with pytest.raises(lb.LBError):
        lb.Solver(2, (8, 8), 0.1, 0.1, 0.1, relax={"s1": 2.5, "s2x": 1, "s22": 1, "w1": 0.1, "wd": 0.01})
    s = lb.Solver(2, (8, 8), 0.02, 1 / 8, 0.01)
    with pytest.raises(lb.LBError) as ei:
        s.step(1)
    assert ei.value.status == lb.LB_ESTATE
    bad = torch.ones((8, 8), dtype=torch.float64, device="cuda")
    bad[3, 4] = -1.0
    with pytest.raises(lb.LBError) as ei:
        s.set_theta0(bad)
    assert ei.value.status == lb.LB_ENONPOS
    bad[3, 4] = float("nan")
    with pytest.raises(lb.LBError) as ei:
        s.set_theta0(bad)
    assert ei.value.status == lb.LB_ENONPOS
    with pytest.raises(ValueError):
        s.set_theta0(torch.ones(7, dtype=torch.float64, device="cuda"))
    # fixed point: a gradient too steep for the fixed-point range
    fx = lb.Solver(2, (8, 8), 0.02, 1 / 8, 0.01, precision="fx64")
    steep = torch.zeros((2, 8, 8), dtype=torch.float64, device="cuda")
    steep[0, 2, 2] = 1e30
    with pytest.raises(lb.LBError) as ei:
        fx.set_theta0(torch.ones((8, 8), dtype=torch.float64, device="cuda"), steep)
    assert ei.value.status == lb.LB_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "fx64", "fp32s"])
def test_graph_replay_matches_direct_launches(precision):
    """lb_step(70) replays two recorded 32-sweep graphs plus 6 launches; it must
    equal 70 single-step calls bit for bit."""
    d, N = 2, (70, 45)
    prob, dx, dt = _problem(d, N, 13)
    out = []
    for chunks in ([70], [1] * 70):
        s = lb.Solver(d, N, prob.nu, dx, dt, precision=precision, theta_ref=1.5)
        s.set_theta0(_dev(prob.theta(N, dx)), _dev(prob.grad(N, dx)))
        for c in chunks:
            s.step(c)
        assert s.nsteps == 70
        out.append(s.macros())
    torch.cuda.synchronize()
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)


def test_steps_captured_into_a_caller_graph():
    """While the caller captures its stream, lb_step launches directly so the
    sweeps become part of the caller's CUDA graph; replaying it advances the
    state exactly like direct stepping."""
    d, N = 2, (64, 48)
    prob, dx, dt = _problem(d, N, 19)
    th0, g0 = _dev(prob.theta(N, dx)), _dev(prob.grad(N, dx))
    ref = lb.Solver(d, N, prob.nu, dx, dt)
    ref.set_theta0(th0, g0)
    ref.step(40)
    th_ref, _, u_ref = ref.macros()
    cap = torch.cuda.Stream()
    s = lb.Solver(d, N, prob.nu, dx, dt, stream=cap)
    s.set_theta0(th0, g0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        s.step(40)  # even: the buffers return to the starting parity
    g.replay()
    torch.cuda.synchronize()
    th, _, u = s.macros()
    torch.cuda.synchronize()
    assert torch.equal(th, th_ref) and torch.equal(u, u_ref)


@pytest.mark.parametrize("precision", ["fp64", "fx64", "fp32s"])
def test_set_viscosity_equals_a_new_context(precision):
    """lb_set_viscosity re-derives Eq. (Bur-Sol) in place: a context made at
    nu1 and moved to nu2 steps exactly like one made at nu2 (also across a
    change between steps, where recorded sweeps must be dropped)."""
    d, N = 2, (70, 45)
    prob, dx, dt = _problem(d, N, 17)
    th0, g0 = _dev(prob.theta(N, dx)), _dev(prob.grad(N, dx))
    a = lb.Solver(d, N, 0.013, dx, dt, precision=precision, theta_ref=1.5)
    a.set_viscosity(prob.nu)
    b = lb.Solver(d, N, prob.nu, dx, dt, precision=precision, theta_ref=1.5)
    assert a.params == b.params
    for s in (a, b):
        s.set_theta0(th0, g0)
        s.step(40)
    a.set_viscosity(0.031)
    a.step(40)
    a.set_viscosity(prob.nu)
    a.step(33)
    b.set_viscosity(0.031)
    b.step(40)
    b.set_viscosity(prob.nu)
    for _ in range(33):
        b.step(1)
    for x, y in zip(a.macros(), b.macros()):
        assert torch.equal(x, y)
    with pytest.raises(lb.LBError) as ei:
        a.set_viscosity(-1.0)
    assert ei.value.status == lb.LB_EINVAL


def test_macros_reports_nonpositive_theta_itself():
    """lb_macros reads back its own flag: a state whose theta is negative
    somewhere is reported by that call (LB_ENONPOS), not by a later one."""
    d, N = 2, (64, 40)
    prob, dx, dt = _problem(d, N, 3)
    s = lb.Solver(d, N, prob.nu, dx, dt)
    s.set_theta0(_dev(prob.theta(N, dx)), _dev(prob.grad(N, dx)))
    s.step(3)
    s.macros()
    snap = s.save_state()
    vals = snap.view(torch.float64)
    pitch, slab, _ = s.state_layout()
    vals[5 * pitch + 7] = -50.0  # rest population of one node (population 0)
    s.load_state(snap, 3)
    with pytest.raises(lb.LBError) as ei:
        s.macros()
    assert ei.value.status == lb.LB_ENONPOS
    s.check()  # reported once, then cleared
    s.set_theta0(_dev(prob.theta(N, dx)), _dev(prob.grad(N, dx)))
    s.macros()


# Rates inside (0, 2) with weights that make the scheme unstable: the largest
# |eigenvalue| of one step's Fourier symbol is 1.34 on this grid.
UNSTABLE = {"s1": 1.46, "s2x": 1.07, "s22": 0.69, "w1": 0.29, "wd": -0.01}


def test_fx64_range_overflow_is_reported_not_wrapped():
    """An unstable custom relaxation set grows the state geometrically.  FX64
    stores int64 values: the sweep flags |f| >= 2^61 and lb_macros reports
    LB_EINVAL instead of returning wrapped values; the context then refuses
    to step until a new state is set.  FP64 reaches non-finite theta
    (LB_ENONPOS) on the same set."""
    d, N = 2, (40, 30)
    prob, dx, dt = _problem(d, N, 11)
    th0, g0 = _dev(prob.theta(N, dx)), _dev(prob.grad(N, dx))
    fx = lb.Solver(d, N, prob.nu, dx, dt, relax=UNSTABLE, precision="fx64")
    fx.set_theta0(th0, g0)
    fx.step(20)
    fx.macros()  # still in range after 20 steps
    fx.step(400)
    with pytest.raises(lb.LBError) as ei:
        fx.macros()
    assert ei.value.status == lb.LB_EINVAL
    with pytest.raises(lb.LBError) as ei:
        fx.step(1)
    assert ei.value.status == lb.LB_ESTATE
    fx.set_theta0(th0, g0)  # a new state clears it
    fx.step(5)
    fx.check()
    fx.step(400)
    with pytest.raises(lb.LBError) as ei:
        fx.sum_theta()
    assert ei.value.status == lb.LB_EINVAL
    f64 = lb.Solver(d, N, prob.nu, dx, dt, relax=UNSTABLE, precision="fp64")
    f64.set_theta0(th0, g0)
    f64.step(3000)
    with pytest.raises(lb.LBError) as ei:
        f64.macros()
    assert ei.value.status == lb.LB_ENONPOS


@pytest.mark.parametrize("precision", ["fp64", "fx64", "fp32s"])
@pytest.mark.parametrize("N,blk", [((70, 45), (4, 24, 512)), ((130, 33), (3, 40, 256)), ((64, 64), (8, 20, 1024)),
                                   ((5, 9), (2, 4, 256)), ((200, 17), (12, 30, 512))])
def test_blocked_sweeps_equal_single_sweeps(N, blk, precision):
    """lb_set_blocking (K steps per launch in shared memory) gives the same
    state bit for bit as one sweep per launch, over remainder launches,
    recorded graphs of 16 launches, a viscosity change in between and a
    return to one sweep per launch."""
    d = 2
    prob, dx, dt = _problem(d, N, 23)
    th0, g0 = _dev(prob.theta(N, dx)), _dev(prob.grad(N, dx))
    out = []
    for mode in ("blocked", "single"):
        s = lb.Solver(d, N, prob.nu, dx, dt, precision=precision, theta_ref=1.5)
        if mode == "blocked":
            s.set_blocking(*blk)
            assert s.blocking()["steps_per_launch"] == blk[0]
        s.set_theta0(th0, g0)
        s.step(16 * blk[0] + 3)
        s.set_viscosity(0.027)
        s.step(7)
        if mode == "blocked":
            s.set_blocking(0)
        s.step(2)
        assert s.nsteps == 16 * blk[0] + 12
        out.append(s.macros())
        s.check()
    torch.cuda.synchronize()
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)


def test_blocking_refused_where_not_built_and_autotune():
    prob, dx, dt = _problem(3, (20, 12, 10), 3)
    s3 = lb.Solver(3, (20, 12, 10), prob.nu, dx, dt)
    with pytest.raises(lb.LBError) as ei:
        s3.set_blocking(4, 16, 512)
    assert ei.value.status == lb.LB_EINVAL
    prob, dx, dt = _problem(2, (96, 80), 3)
    s = lb.Solver(2, (96, 80), prob.nu, dx, dt, precision="fx64", boundary=["mirror", "periodic"])
    with pytest.raises(lb.LBError) as ei:
        s.set_blocking(4, 16, 512)
    assert ei.value.status == lb.LB_EINVAL
    s = lb.Solver(2, (96, 80), prob.nu, dx, dt, precision="fx64")
    with pytest.raises(lb.LBError) as ei:
        s.set_blocking(8, 300, 512)  # tile plus halo beyond shared memory
    assert ei.value.status == lb.LB_EINVAL
    choice = s.autotune(8)
    assert choice["steps_per_launch"] in (0, 2, 3, 4, 5, 6, 8, 12) and choice["us_per_step"] > 0
    with pytest.raises(lb.LBError) as ei:
        s.step(1)  # the trials overwrote the state
    assert ei.value.status == lb.LB_ESTATE
    s.set_theta0(_dev(prob.theta((96, 80), dx)), _dev(prob.grad((96, 80), dx)))
    s.step(5)
    s.macros()


def test_blocked_fx64_range_overflow_is_reported():
    """The blocked FX64 sweep checks the values it stores: an unstable
    relaxation set is reported (LB_EINVAL), not wrapped."""
    d, N = 2, (40, 30)
    prob, dx, dt = _problem(d, N, 11)
    fx = lb.Solver(d, N, prob.nu, dx, dt, relax=UNSTABLE, precision="fx64")
    fx.set_blocking(4, 16, 256)
    fx.set_theta0(_dev(prob.theta(N, dx)), _dev(prob.grad(N, dx)))
    fx.step(20)
    fx.macros()
    fx.step(400)
    with pytest.raises(lb.LBError) as ei:
        fx.macros()
    assert ei.value.status == lb.LB_EINVAL
