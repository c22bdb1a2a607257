"""Benchmark: MLUPS and fraction of the HBM roofline of the MRT-LB hot path.

Workload (default): 2D D2Q9, periodic 4096^2, nu = 0.02, eps = 0.2048,
theta0 = 2 + sin(2 pi x) sin(2 pi y) (the 2D sine family), FP64 and FP32
shifted storage.  One benchmark step is one pass of the whole hot path:
lb_set_theta0 (initialisation), S fused pull-stream + collide sweeps,
lb_macros (theta, grad theta, u), lb_sum_theta and lb_reduce (error norms
against the closed-form solution at t = S dt).  MLUPS = nodes * S / time.

The state (2 x 1.2 GB for FP64) is larger than L2 (129 MB), so there is no
L2 flush between steps.  Times come from CUDA events on the solver's
stream.  ``e2e`` repeats the step through the public API from pinned host
buffers (inputs copied in, theta and u copied out, inside the timed
region).  ``--impl reference`` times the FP64 CPU oracle instead.

Precisions: the headline is FX64 (64-bit fixed-point state, exact integer
moment sums; FP64-accurate and HBM-bound on GB300, whose FP64 pipe runs at
1/64 of FP32); FP64 and FP32-shifted are reported under ``variants``.
Also reported: ``batched`` (512 uneven 2D instances x 2000 steps),
``adjoint`` (512^2, T = 2000: reverse-step cost and finite-difference
checks) and ``sweeps_3d`` (D3Q19 256^3).  ``--accuracy`` prints the
error-vs-exact convergence table instead.

Multi-GPU: the path is one periodic grid per GPU; ranks run independent
replicas (weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2309_02825_gb300 import workloads as W  # noqa: E402

METRIC = "MLUPS and % of HBM BW vs L2 err to exact: FP64 vs FP32-shifted; adjoint step cost"
UNIT = "MLUPS"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fx64", choices=["fx64", "fp64", "fp32s"],
                   help="headline precision; the other two are reported as variants")
    p.add_argument("--N", type=int, default=4096)
    p.add_argument("--sweeps", type=int, default=100, help="sweeps per benchmark step")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--slab", action="store_true",
                   help="one N^2 FX64 grid cut into one slab per rank (ghost-layer exchange every step) instead of "
                        "independent replicas: strong scaling")
    p.add_argument("--no-blocking", action="store_true",
                   help="one sweep per launch only (skip the autotuner's blocked candidates)")
    p.add_argument("--no-variant", action="store_true", help="skip the other precisions' sub-results")
    p.add_argument("--no-batched", action="store_true", help="skip the batched 512-instance measurement")
    p.add_argument("--no-adjoint", action="store_true", help="skip the 512^2 adjoint measurement")
    p.add_argument("--no-3d", action="store_true", help="skip the 3D 256^3 sweep measurement")
    p.add_argument("--no-4d", action="store_true", help="skip the 4D D4Q33 50^4 measurement")
    p.add_argument("--no-walls", action="store_true", help="skip the mirror-wall measurements (Example 1)")
    p.add_argument("--accuracy", action="store_true",
                   help="print the error-vs-exact convergence table (1D, 2D up to 4096^2, 3D up to 256^3) and exit")
    p.add_argument("--accuracy-precisions", default="fp64,fx64,fp32s")
    p.add_argument("--profile-batch", default=None, metavar="COUNT,STEPS[,PREC[,K,TILE,THREADS]]",
                   help="minimal command for ncu: COUNT batched 2D instances, STEPS steps, then exit")
    p.add_argument("--profile-adjoint", default=None, metavar="PREC,N,T",
                   help="minimal command for ncu: forward + seed + T reverse steps at N^2, then exit")
    p.add_argument("--profile-sweep", default=None, metavar="D,PREC,N,STEPS",
                   help="run STEPS sweeps of one D-dimensional N^D grid at PREC and exit (for ncu captures)")
    p.add_argument("--blocking", default=None, metavar="K,TILE,THREADS",
                   help="blocked sweeps of K steps per launch for the headline step (instead of the autotuner's "
                        "pick) or for --profile-sweep")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_sha():
    """sha256 (16 hex digits) of the sweep kernels' sources with comments and
    whitespace removed, so that only a change of code voids a capture."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2309_02825_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("lb_internal.cuh", "lb_device.cuh", "lb_kernels.cu", "lb_fx.cu"):
        text = open(os.path.join(csrc, name)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def blocked_source_sha():
    """sha256 (16 hex digits) of the blocked kernel's sources (comments and
    whitespace removed)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2309_02825_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("lb_internal.cuh", "lb_device.cuh", "lb_batch.cu"):
        text = open(os.path.join(csrc, name)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profile_blocked(kernel_key):
    """(warp instructions, DRAM bytes) per launch of a blocked configuration,
    from a committed ncu summary of the same kernel source; (None, None) if
    the kernel changed since or the configuration was not captured."""
    try:
        sha = blocked_source_sha()
        for line in open(os.path.join(ROOT, "profiles", "blocked.txt")):
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel_key and parts[1] == sha:
                return float(parts[2]), float(parts[3])
    except OSError:
        pass
    return None, None


def blocked_launch_bytes(N0, N1, K, tile, elem, q=9):
    """HBM bytes one blocked launch must move: every tile read with its
    K-node halo and written once."""
    return blocked_bytes_per_lu([(N0, N1)], K, tile, elem, q) * N0 * N1 * K


def profile_fp64_inst(kernel_key):
    """FP64 instructions per lattice update (thread-level, i.e. 32 x the warp
    instructions ncu counts in sm__inst_executed_pipe_fp64.sum, per node) of a
    sweep, from a committed ncu summary; valid only while the kernel source is
    unchanged (same sha)."""
    try:
        sha = kernel_source_sha()
        for line in open(os.path.join(ROOT, "profiles", "fp64_inst.txt")):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel_key and parts[1] == sha:
                return float(parts[2])
    except OSError:
        pass
    return None


def profile_traffic(kernel_key):
    """DRAM bytes per launch from a committed ncu summary for this kernel,
    valid only while the kernel source is unchanged (same sha)."""
    try:
        sha = kernel_source_sha()
        path = os.path.join(ROOT, "profiles", "traffic.txt")
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel_key and parts[1] == sha:
                return float(parts[2])
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce(v, op):
    """All-reduce one float over the process group (CUDA tensor for NCCL,
    CPU tensor for gloo)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def barrier_max(t, world):
    """Slowest rank's time (the job finishes when the last replica does)."""
    if world == 1:
        return t
    import torch.distributed as dist
    return _reduce(t, dist.ReduceOp.MAX)


def aggregate(units, seconds, world):
    """Whole-job throughput of independent replicas: units summed over ranks
    divided by the slowest rank's time."""
    if world == 1:
        return units / seconds
    import torch.distributed as dist
    return _reduce(units, dist.ReduceOp.SUM) / _reduce(seconds, dist.ReduceOp.MAX)


# ---------------------------------------------------------------------------
# Our implementation.
# ---------------------------------------------------------------------------

def run_ours(args, precision, world, rank, local, peaks, with_e2e, label_main, blocking=True):
    import torch
    from paper_2309_02825_gb300 import lb

    torch.cuda.set_device(local)
    case = W.sine_2d(args.N)
    S = args.sweeps
    N, d = case.N, case.d
    T = S * case.dt
    th0_h = case.problem.theta(N, case.dx)
    g0_h = np.ascontiguousarray(case.problem.grad(N, case.dx))
    ex_t_h = case.problem.theta(N, case.dx, T)
    ex_u_h = np.ascontiguousarray(case.problem.u(N, case.dx, T))
    th0 = torch.from_numpy(th0_h).cuda()
    g0 = torch.from_numpy(g0_h).cuda()
    ex_t = torch.from_numpy(ex_t_h).cuda()
    ex_u = torch.from_numpy(ex_u_h).cuda()

    stream = torch.cuda.Stream()
    theta_ref = 2.0 if precision == "fp32s" else 0.0
    s = lb.Solver(d, N, case.nu, case.dx, case.dt, precision=precision, theta_ref=theta_ref, stream=stream)
    # one sweep per launch, or K sweeps per launch in shared memory: the
    # autotuner times both on this grid (outside the timed region)
    with torch.cuda.stream(stream):
        if blocking and args.blocking and label_main:
            # pinned (K, tile, threads): the autotuner's timings are not
            # trustworthy under a profiler, so profiled runs pin its pick
            k_, t_, th_ = (int(v) for v in args.blocking.split(","))
            s.set_blocking(k_, t_, th_)
            tune = {"steps_per_launch": k_, "tile": t_, "threads": th_, "pinned": True}
        elif blocking and not args.no_blocking:
            tune = s.autotune(24)
        else:
            tune = {"steps_per_launch": 0}
    K = tune["steps_per_launch"]
    th = torch.empty(tuple(reversed(N)), dtype=torch.float64, device="cuda")
    gr = torch.empty((d,) + tuple(reversed(N)), dtype=torch.float64, device="cuda")
    u = torch.empty_like(gr)

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    out = {}

    def one_step(i=None):
        s.set_theta0(th0, g0)
        if i is not None:
            ev_s[i].record(stream)
        s.step(S)
        if i is not None:
            ev_e[i].record(stream)
        s.macros(th, gr, u)
        out["total"] = s.sum_theta()
        out["norms"] = s.reduce(th, u, ex_t, ex_u)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local) if label_main else None
    if clocks:
        clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for i in range(args.steps):
            one_step(i)
        t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    elapsed_local = t_start.elapsed_time(t_end) / 1e3
    sweep_ms = sum(a.elapsed_time(b) for a, b in zip(ev_s, ev_e)) / (args.steps * S)

    nodes = case.nodes
    value = aggregate(nodes * S * args.steps, elapsed_local, world) / 1e6
    elapsed = barrier_max(elapsed_local, world)
    q = 9
    elem = 4 if precision == "fp32s" else 8
    bytes_lu = 2 * q * elem
    norms = out["norms"]
    ctype = {"fp64": "double", "fp32s": "float", "fx64": "long long"}[precision]
    sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if K == 0:
        # one sweep per launch: HBM-bound, 2 q sizeof(T) bytes per update
        achieved = bytes_lu * nodes / (sweep_ms / 1e3) / 1e9
        roofline = {
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"],
            "traffic": profile_traffic("sweep_d2q9_%s_%d" % (precision, args.N)),
            "kernel": "sweep_kernel<D2Q9,%s>" % ctype,
            "algorithmic_bytes_per_launch": bytes_lu * nodes,
            "peak_source": peaks["source"],
        }
    else:
        # blocked: K sweeps per launch in shared memory, bound by instruction
        # issue (4 warp instructions per SM per clock); its HBM traffic is the
        # tiles with their halos
        launch_s = sweep_ms / 1e3 * K
        key = "blocked_d2q9_%s_%d_K%d_T%d_TH%d" % (precision, args.N, K, tune["tile"], tune["threads"])
        inst, dram = profile_blocked(key)
        peak_issue = 4 * sms * sm_mhz * 1e6 / 1e9
        ach_issue = None if inst is None else inst / launch_s / 1e9
        blk_bytes = blocked_launch_bytes(N[0], N[1], K, tune["tile"], elem)
        roofline = {
            "bound": "alu", "achieved": ach_issue, "peak": peak_issue, "unit": "G warp-inst/s",
            "frac": None if ach_issue is None else ach_issue / peak_issue,
            "traffic": dram,
            "kernel": "batch_tb_kernel<D2Q9,%s,%d> (%d sweeps per launch, tiles of %d)" % (
                ctype, tune["threads"], K, tune["tile"]),
            "warp_inst_per_launch": inst, "sms": sms, "sm_mhz": sm_mhz,
            "peak_source": "4 warp instructions per SM per clock x SMs x sampled SM clock",
            "algorithmic_bytes_per_launch": blk_bytes,
            "hbm_gbs_of_algorithmic_bytes": blk_bytes / launch_s / 1e9,
            "hbm_frac_of_algorithmic_bytes": blk_bytes / launch_s / 1e9 / peaks["hbm_gbs"],
            "per_step_equivalent_hbm_frac": bytes_lu * nodes / (sweep_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "counters_source": "profiles/blocked.txt (ncu at this size, same kernel source)",
        }
    res = {
        "value": value,
        "ms_per_step": elapsed / args.steps * 1e3,
        "sweep_ms": sweep_ms,
        "bytes_per_lu": bytes_lu,
        "blocking": tune,
        "roofline": roofline,
        "error": {"t": T, "theta_rmse": norms["theta"]["rmse"],
                  "u_rmse": math.sqrt(sum(norms["u%d" % a]["rmse"] ** 2 for a in range(d)) / d),
                  "u_linf": max(norms["u%d" % a]["linf"] for a in range(d)),
                  "u_rel_l2": math.sqrt(sum(norms["u%d" % a]["rel_l2"] ** 2 for a in range(d)) / d),
                  "sum_theta_drift": abs(out["total"] - float(th0_h.sum())) / float(th0_h.sum())},
        "clocks": clk,
        "gpu_launches": args.steps * ((S // K + (1 if S % K else 0) if K else S) + 6 + (2 if precision == "fx64" else 0)),
    }
    if precision == "fp64" and K == 0:
        # The FP64 sweep is bound by the FP64 pipe: GB300 issues 2 FP64 lane
        # operations per SM per clock (1/64 of FP32).  The instructions per
        # update come from an ncu capture of this kernel source (null when the
        # kernel changed since), the SM count from the device.
        peak_inst = sms * 2 * sm_mhz * 1e6 / 1e9
        ipl = profile_fp64_inst("sweep_d2q9_fp64")
        ach_inst = None if ipl is None else ipl * nodes / (sweep_ms / 1e3) / 1e9
        res["roofline_fp64_pipe"] = {"bound": "alu", "achieved": ach_inst, "peak": peak_inst,
                                     "unit": "G FP64 lane-ops/s",
                                     "frac": None if ach_inst is None else ach_inst / peak_inst,
                                     "fp64_inst_per_lu": ipl, "sms": sms, "sm_mhz": sm_mhz,
                                     "fp64_inst_source": "profiles/fp64_inst.txt (ncu sm__inst_executed_pipe_fp64)"}

    if with_e2e:
        res["e2e"] = run_e2e(args, s, case, th0_h, g0_h, ex_t_h, ex_u_h, stream, world)
    s.close()
    return res


def run_e2e(args, s, case, th0_h, g0_h, ex_t_h, ex_u_h, stream, world):
    """The same step through the public API from pinned host buffers: every
    step uploads its inputs (theta0, grad theta0 and the exact fields the
    error norms are taken against) and reads its result, the error norms
    that lb_reduce returns to the host, all inside the timed region.  The
    uploads are double buffered on a second stream, so step k+1's inputs move
    while step k computes; events order each copy against the solver.  The
    exact fields, which only the error norms read, are uploaded after theta0
    and its gradient, so a step starts before they have arrived."""
    import torch
    S = args.sweeps
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [pin(th0_h), pin(g0_h), pin(ex_t_h), pin(ex_u_h)]
    d_in = [[torch.empty_like(h, device="cuda") for h in h_in] for _ in range(2)]
    shape = tuple(reversed(case.N))
    d_out = (torch.empty(shape, dtype=torch.float64, device="cuda"),
             torch.empty((case.d,) + shape, dtype=torch.float64, device="cuda"))
    cs = torch.cuda.Stream()
    in_ready = [torch.cuda.Event() for _ in range(2)]  # theta0 and its gradient: needed first
    ex_ready = [torch.cuda.Event() for _ in range(2)]  # the exact fields: needed by the norms at the end
    solved = [torch.cuda.Event() for _ in range(2)]
    results = []

    def h2d(b):
        with torch.cuda.stream(cs):
            cs.wait_event(solved[b])  # the step that last used these inputs is done
            for i, (h, dv) in enumerate(zip(h_in, d_in[b])):
                dv.copy_(h, non_blocking=True)
                if i == 1:
                    in_ready[b].record(cs)
            ex_ready[b].record(cs)

    def run(n):
        for b in range(2):
            solved[b].record(cs)
        h2d(0)
        for k in range(n):
            b = k % 2
            if k + 1 < n:
                h2d(1 - b)
            stream.wait_event(in_ready[b])
            with torch.cuda.stream(stream):
                s.set_theta0(d_in[b][0], d_in[b][1])
                s.step(S)
                s.macros(d_out[0], None, d_out[1])
                stream.wait_event(ex_ready[b])
                results.append(s.reduce(d_out[0], d_out[1], d_in[b][2], d_in[b][3]))  # read back to the host
                solved[b].record(stream)
        torch.cuda.synchronize()

    run(max(1, args.warmup))
    t0 = time.perf_counter()
    run(args.steps)
    el = time.perf_counter() - t0
    value = aggregate(case.nodes * S * args.steps, el, world) / 1e6
    h2d_b = sum(h.numel() * h.element_size() for h in h_in)
    d2h_b = 8 * (3 * (case.d + 1) + 1)  # lb_reduce's norms and sum, FP64
    # the upload rate on its own (outside the timed region): the first upload
    # of the timed run cannot overlap any compute
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(cs):
        e0.record(cs)
        for h, dv in zip(h_in, d_in[0]):
            dv.copy_(h, non_blocking=True)
        e1.record(cs)
    torch.cuda.synchronize()
    h2d_ms = e0.elapsed_time(e1)
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
            "overlap": "uploads double-buffered on a second stream; the result read is the step's error norms",
            "copy_rates": {"h2d_gbs": h2d_b / h2d_ms / 1e6, "unoverlapped_ms_per_run": h2d_ms, "steps": args.steps},
            "u_rmse_last_step": results[-1]["u0"]["rmse"]}


def blocked_bytes_per_lu(sizes, K, tile, elem, q=9):
    """HBM bytes per lattice update of blocked launches (K steps each): every
    tile is read with its K-node halo and written once per launch, tiles cut
    as the library cuts them (ceil(N / tile) near-equal tiles per axis)."""
    moved, lus = 0, 0
    for n0, n1 in sizes:
        ntx, nty = -(-n0 // tile), -(-n1 // tile)
        tx, ty = -(-n0 // ntx), -(-n1 // nty)
        for y0 in range(0, n1, ty):
            for x0 in range(0, n0, tx):
                w, h = min(tx, n0 - x0), min(ty, n1 - y0)
                moved += q * elem * ((w + 2 * K) * (h + 2 * K) + w * h)
                lus += w * h * K
    return moved / lus


def run_batched(local):
    """512 independent 2D instances (N log-uniform in [32, 512], nu log-uniform
    in [0.005, 0.1], dt = 4 dx^2), FP32 shifted, 2000 steps: the autotuned
    schedule (blocked launches of K steps in shared memory, or one launch per
    step) vs one launch per instance per step vs one flat launch per step."""
    import torch
    from paper_2309_02825_gb300 import lb

    torch.cuda.set_device(local)
    cases = W.batched_2d(512, nsteps=2000)
    sizes = [c.N for c in cases]
    th0 = np.concatenate([c.problem.theta(c.N, c.dx).ravel() for c in cases])
    g0 = np.concatenate([np.ascontiguousarray(c.problem.grad(c.N, c.dx)).ravel() for c in cases])
    stream = torch.cuda.Stream()
    b = lb.Batch(sizes, [c.nu for c in cases], [c.dx for c in cases], [c.dt for c in cases],
                 precision="fp32s", theta_ref=[1.5] * len(cases), stream=stream)
    choice = b.autotune(10)
    th0_d, g0_d = torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda()
    nodes = b.total_nodes
    steps = cases[0].nsteps

    def timed(n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            b.set_theta0(th0_d, g0_d)
            b.step(64)  # warm-up (graphs recorded, L2 warm)
            b.set_theta0(th0_d, g0_d)
            e0.record(stream)
            b.step(n)
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    t_tuned = timed(steps)
    sched = b.schedule()
    with torch.cuda.stream(stream):
        th, u = b.macros()
        ex_t = np.concatenate([c.problem.theta(c.N, c.dx, c.t_end).ravel() for c in cases])
        ex_u = np.concatenate([np.ascontiguousarray(c.problem.u(c.N, c.dx, c.t_end)).ravel() for c in cases])
        err = b.errors(th, u, torch.from_numpy(ex_t).cuda(), torch.from_numpy(ex_u).cuda())
    base_steps = 20
    b.set_schedule(0.0, 256, False)
    t_base = timed(base_steps) * steps / base_steps
    b.set_schedule(1e18, 256, True)
    t_flat = timed(base_steps * 10) * steps / (base_steps * 10)
    b.close()
    lu = nodes * steps
    # the same workload in 64-bit fixed point (FP64-grade accuracy, 144 B per update)
    bx = lb.Batch(sizes, [c.nu for c in cases], [c.dx for c in cases], [c.dt for c in cases], precision="fx64",
                  stream=stream)
    choice_fx = bx.autotune(10)
    ex0, ex1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        bx.set_theta0(th0_d, g0_d)
        bx.step(64)
        bx.set_theta0(th0_d, g0_d)
        ex0.record(stream)
        bx.step(steps)
        ex1.record(stream)
        thx, ux = bx.macros()
        errx = bx.errors(thx, ux, torch.from_numpy(ex_t).cuda(), torch.from_numpy(ex_u).cuda())
    torch.cuda.synchronize()
    t_fx = ex0.elapsed_time(ex1) / 1e3
    bx.close()
    peak = load_peaks()["hbm_gbs"]

    def roof(choice, t, elem):
        """Per-step-equivalent fraction (2 q elem bytes per update, what one
        launch per step must move) and, for blocked launches, the fraction of
        the bytes they do move."""
        out = {"per_step_equivalent_hbm_frac": 2 * 9 * elem * lu / t / 1e9 / peak}
        if choice["steps_per_launch"]:
            bpl = blocked_bytes_per_lu(sizes, choice["steps_per_launch"], choice["tile"], elem)
            out.update({"blocked_bytes_per_lu": bpl, "blocked_hbm_gbs": bpl * lu / t / 1e9,
                        "blocked_hbm_frac": bpl * lu / t / 1e9 / peak})
        return out

    fx64 = {"aggregate_mlups": lu / t_fx / 1e6, "instances_per_s": len(cases) / t_fx, "seconds": t_fx,
            "autotune": choice_fx, **roof(choice_fx, t_fx, 8),
            "u_rmse_max_over_instances": float(np.max(errx[:, 1])),
            "theta_rmse_max_over_instances": float(np.max(errx[:, 0]))}
    return {
        "workload": "512 x 2D D2Q9, N log-uniform [32,512], nu log-uniform [0.005,0.1], dt=4dx^2, fp32 shifted, "
                    "2000 steps",
        "instances": len(cases), "total_nodes": nodes, "steps": steps,
        "instances_per_s": len(cases) / t_tuned, "aggregate_mlups": lu / t_tuned / 1e6, "seconds": t_tuned,
        "schedule": sched,
        "autotune": choice,
        "one_launch_per_instance": {"aggregate_mlups": lu / t_base / 1e6, "instances_per_s": len(cases) / t_base,
                                    "sample_steps": base_steps},
        "flat_one_group": {"aggregate_mlups": lu / t_flat / 1e6, "sample_steps": 10 * base_steps},
        "speedup_vs_one_launch_per_instance": t_base / t_tuned,
        "u_rmse_max_over_instances": float(np.max(err[:, 1])),
        "theta_rmse_max_over_instances": float(np.max(err[:, 0])),
        **roof(choice, t_tuned, 4),
        "fx64": fx64,
    }


def run_adjoint(local, precision="fp64"):
    """Adjoint cost at 512^2, T = 2000, sqrt(T) checkpoints: forward with
    checkpoints, reverse pass with segment recompute, per-step cost against a
    plain forward sweep, and central-difference checks of dL/dtheta0 along 16
    seeded random directions and of dL/dnu (FP64 and FX64)."""
    import torch
    from paper_2309_02825_gb300 import lb

    torch.cuda.set_device(local)
    case = W.adjoint_2d(512, 2000)
    N, d, T = case.N, case.d, case.nsteps
    th0 = torch.from_numpy(case.problem.theta(N, case.dx)).cuda()
    ut = torch.from_numpy(np.ascontiguousarray(case.extra["target"].u(N, case.dx, T * case.dt))).cuda()
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def grad(nu, th, timed=False):
        s = lb.Solver(d, N, nu, case.dx, case.dt, precision=precision, stream=stream)
        a = lb.Adjoint(s, T, checkpoint=0, want_nu=True)
        with torch.cuda.stream(stream):
            if timed:
                ev[0].record(stream)
            u = a.forward(th)
            if timed:
                ev[1].record(stream)
            r = u - ut
            a.seed(r)
            a.step(T)
            g, dnu = a.result()
            if timed:
                ev[2].record(stream)
            L = 0.5 * float((r * r).sum())
        info = a.info()
        a.close()
        s.close()
        return L, g, dnu, info

    ls = lb.Solver(d, N, case.nu, case.dx, case.dt, precision=precision, stream=stream)
    u_buf = torch.empty((d,) + tuple(reversed(N)), dtype=torch.float64, device="cuda")

    def loss(nu, th):
        """The forward map the adjoint differentiates (theta0 with its FD4
        gradient, T sweeps, u), on one reused context."""
        with torch.cuda.stream(stream):
            ls.set_viscosity(nu)
            ls.set_theta0(th.contiguous())
            ls.step(T)
            ls.macros(u=u_buf, want=("u",))
            r = u_buf - ut
            L = 0.5 * float((r * r).sum())
        return L

    grad(case.nu, th0)  # warm-up
    L, g, dnu, info = grad(case.nu, th0, timed=True)
    torch.cuda.synchronize()
    t_fwd = ev[0].elapsed_time(ev[1]) / 1e3
    t_bwd = ev[1].elapsed_time(ev[2]) / 1e3
    # plain forward sweep time at this size
    s = lb.Solver(d, N, case.nu, case.dx, case.dt, precision=precision, stream=stream)
    with torch.cuda.stream(stream):
        s.set_theta0(th0)
        s.step(50)
        ev[3].record(stream)
        s.step(T)
        ev[4].record(stream)
    torch.cuda.synchronize()
    t_sweep = ev[3].elapsed_time(ev[4]) / 1e3 / T
    s.close()
    # central differences on 16 seeded random directions (FP64 and FX64; the
    # FP32s forward map is only float-accurate, too coarse for a difference)
    rng = np.random.default_rng(2314)
    checks = []
    fd_nu = float("nan")
    if precision in ("fp64", "fx64"):
        for _ in range(16):
            v = torch.from_numpy(rng.normal(size=tuple(th0.shape))).cuda()
            h = 1e-5
            fd = (loss(case.nu, th0 + h * v) - loss(case.nu, th0 - h * v)) / (2 * h)
            checks.append(abs(float((g * v).sum()) / fd - 1.0))
        hn = 1e-6 * case.nu
        fd_nu = (loss(case.nu + hn, th0) - loss(case.nu - hn, th0)) / (2 * hn)
    ls.close()
    return {
        "workload": "2D D2Q9 512^2, nu=0.02, eps=0.2048, T=2000, L=0.5||u(T)-u_target||^2, %s, checkpoint every %d "
                    "steps (%d checkpoints)" % (precision, info["checkpoint"], info["checkpoints"]),
        "forward_with_checkpoints_s": t_fwd, "reverse_s": t_bwd, "plain_sweep_us": t_sweep * 1e6,
        "reverse_step_us": t_bwd / T * 1e6,
        "adjoint_step_cost_vs_forward_step": t_bwd / T / t_sweep,
        "gradient_total_cost_vs_forward": (t_fwd + t_bwd) / (T * t_sweep),
        "loss": L, "dL_dnu": dnu, "fd_rel_err_theta0_dirs": checks, "fd_rel_err_nu": abs(dnu / fd_nu - 1.0),
        "workspace_bytes": info["bytes"],
        # per reverse step: the reverse kernel reads lambda_{n+1} and f_n and writes lambda_n (q values each per
        # node), and the segment recompute runs one forward sweep (reads and writes q values per node)
        "algorithmic_bytes_per_reverse_step": _adj_bytes(case, precision)[0],
        "bytes_vs_forward_step": _adj_bytes(case, precision)[0] / _adj_bytes(case, precision)[1],
    }


def _adj_bytes(case, precision):
    """(algorithmic bytes of one reverse step incl. its recompute sweep, of one forward sweep)."""
    q, nodes = 1 + 2 * case.d * case.d, int(np.prod(case.N))
    es = 4 if precision == "fp32s" else 8  # stored state value
    ea = 4 if precision == "fp32s" else 8  # adjoint field value (float, int64 fixed point or double)
    fwd = 2 * q * es * nodes
    return (2 * q * ea + q * es) * nodes + fwd, fwd


def run_slab(args, world, rank, local, steps, warmup):
    """One 2D sine grid (args.N^2, FX64) cut along y into one slab per rank;
    every sweep is preceded by the ghost-layer exchange (NCCL point-to-point
    between ranks; with one rank the buffers wrap onto the part itself).
    Returns (whole-grid MLUPS, ms per sweep, bytes sent per rank and sweep)."""
    import torch
    from paper_2309_02825_gb300 import slab as SL
    torch.cuda.set_device(local)
    case = W.sine_2d(args.N)
    N = case.N
    th0 = torch.from_numpy(case.problem.theta(N, case.dx))
    g0 = torch.from_numpy(np.ascontiguousarray(case.problem.grad(N, case.dx)))
    r = SL.SlabRunner(2, N, case.nu, case.dx, case.dt, "fx64", rank=rank, world=world)
    r.set_theta0(th0, g0)
    r.step(warmup)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r.step(steps)
    e1.record()
    torch.cuda.synchronize()
    t = barrier_max(e0.elapsed_time(e1) / 1e3, world)
    sent = 2 * r.slab.halo_count * r.slab.elem
    return {"mlups": N[0] * N[1] * steps / t / 1e6, "ms_per_sweep": t / steps * 1e3, "parts": world,
            "bytes_sent_per_rank_per_sweep": sent, "owned_layers_rank0": r.slab.nz}


def _run_case(case, precision, theta_ref, stream, th0=None, g0=None, nsteps=None, exact=None):
    """Run one workload case to its end time; return the error norms."""
    import torch
    from paper_2309_02825_gb300 import lb
    N, d = case.N, case.d
    n = case.nsteps if nsteps is None else nsteps
    th0 = th0 if th0 is not None else torch.from_numpy(case.problem.theta(N, case.dx)).cuda()
    g0 = g0 if g0 is not None else torch.from_numpy(np.ascontiguousarray(case.problem.grad(N, case.dx))).cuda()
    s = lb.Solver(d, N, case.nu, case.dx, case.dt, precision=precision, theta_ref=theta_ref, stream=stream)
    with torch.cuda.stream(stream):
        s.set_theta0(th0, g0)
        s.step(n)
        th, _, u = s.macros(want=("theta", "u"))
        T = n * case.dt
        if exact is None:
            exact = (torch.from_numpy(case.problem.theta(N, case.dx, T)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(case.problem.u(N, case.dx, T))).cuda())
        r = s.reduce(th, u, exact[0], exact[1])
    s.close()
    return {"theta_rmse": r["theta"]["rmse"],
            "u_rmse": math.sqrt(sum(r["u%d" % a]["rmse"] ** 2 for a in range(d)) / d),
            "u_linf": max(r["u%d" % a]["linf"] for a in range(d)),
            "u_rel_l2": math.sqrt(sum(r["u%d" % a]["rel_l2"] ** 2 for a in range(d)) / d)}


def run_3d(local, peaks):
    """3D D3Q19 periodic 256^3 (the 3D Fourier family): sweep throughput and
    %HBM for each precision, and the error against the exact solution at
    t_end = 0.02 (256 steps)."""
    import torch
    from paper_2309_02825_gb300 import lb
    torch.cuda.set_device(local)
    case = W.fourier_3d(256)
    stream = torch.cuda.Stream()
    th0 = torch.from_numpy(case.problem.theta(case.N, case.dx)).cuda()
    g0 = torch.from_numpy(np.ascontiguousarray(case.problem.grad(case.N, case.dx))).cuda()
    exact = (torch.from_numpy(case.problem.theta(case.N, case.dx, case.t_end)).cuda(),
             torch.from_numpy(np.ascontiguousarray(case.problem.u(case.N, case.dx, case.t_end))).cuda())
    out = {"workload": "3D D3Q19 periodic 256^3, nu=0.01, eps=0.0512, 1.5 + 8 seeded modes, t_end=0.02 (256 steps)"}
    for prec in ("fx64", "fp64", "fp32s"):
        s = lb.Solver(3, case.N, case.nu, case.dx, case.dt, precision=prec, theta_ref=1.5, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            s.set_theta0(th0, g0)
            s.step(10)
            e0.record(stream)
            s.step(50)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 50
        s.close()
        elem = 4 if prec == "fp32s" else 8
        gbs = 2 * 19 * elem * case.nodes / (ms / 1e3) / 1e9
        err = _run_case(case, prec, 1.5, stream, th0, g0, exact=exact)
        out[prec] = {"sweep_ms": ms, "mlups": case.nodes / (ms / 1e3) / 1e6, "bytes_per_lu": 2 * 19 * elem,
                     "hbm_frac": gbs / peaks["hbm_gbs"], "achieved_gbs": gbs, "error_t_end": err,
                     "traffic": profile_traffic("sweep_d3q19_%s_256" % prec)}
    return out


TABLE1 = {  # the paper's Table 1 (Example 1, t = 2): RMSE at levels 0..3, theta then u
    0.5: ((7.8613e-4, 4.8926e-5, 3.0595e-6, 1.9139e-7), (1.9827e-5, 1.1821e-6, 7.2429e-8, 4.4865e-9)),
    1.0: ((2.4232e-4, 1.5014e-5, 9.3770e-7, 5.8641e-8), (3.2184e-5, 2.0194e-6, 1.2608e-7, 7.8713e-9)),
    1.5: ((2.3106e-4, 1.3918e-5, 8.6303e-7, 5.3874e-8), (1.0796e-4, 6.4468e-6, 3.9752e-7, 2.4739e-8)),
    2.0: ((2.1330e-4, 1.2349e-5, 7.5838e-7, 4.7229e-8), (1.8574e-4, 1.0638e-5, 6.4967e-7, 4.0343e-8)),
}


def run_walls(local, peaks):
    """Mirror walls: (1) the 2D FX64 sweep at 4096^2 with walls on both axes
    beside the periodic one; (2) the paper's Example 1 (walls at x = 0, 1)
    through the CUDA path, RMSE and CR per eps and level, with Table 1."""
    import torch
    from paper_2309_02825_gb300 import lb
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    out = {}
    n = 4096
    case = W.sine_2d(n)
    N = (n, n)
    th0 = torch.from_numpy(case.problem.theta(N, case.dx)).cuda()
    g0 = torch.from_numpy(np.ascontiguousarray(case.problem.grad(N, case.dx))).cuda()
    for kind in ("periodic", "mirror"):
        s = lb.Solver(2, N, case.nu, case.dx, case.dt, precision="fx64", stream=stream, boundary=[kind, kind])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            s.set_theta0(th0, g0)
            s.step(10)
            e0.record(stream)
            s.step(100)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 100
        s.close()
        gbs = 2 * 9 * 8 * n * n / (ms / 1e3) / 1e9
        out["sweep_2d_4096_fx64_" + kind] = {"sweep_ms": ms, "mlups": n * n / (ms / 1e3) / 1e6,
                                              "hbm_frac": gbs / peaks["hbm_gbs"]}
    c3 = W.fourier_3d(256)
    th3 = torch.from_numpy(c3.problem.theta(c3.N, c3.dx)).cuda()
    g3 = torch.from_numpy(np.ascontiguousarray(c3.problem.grad(c3.N, c3.dx))).cuda()
    for kind in ("periodic", "mirror"):
        s = lb.Solver(3, c3.N, c3.nu, c3.dx, c3.dt, precision="fx64", stream=stream, boundary=[kind] * 3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            s.set_theta0(th3, g3)
            s.step(10)
            e0.record(stream)
            s.step(50)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 50
        s.close()
        gbs = 2 * 19 * 8 * c3.nodes / (ms / 1e3) / 1e9
        out["sweep_3d_256_fx64_" + kind] = {"sweep_ms": ms, "mlups": c3.nodes / (ms / 1e3) / 1e6,
                                             "hbm_frac": gbs / peaks["hbm_gbs"]}
    ex1 = {}
    for eps in (0.5, 1.0, 1.5, 2.0):
        rows = {"theta": [], "u": []}
        for level in range(4):
            c = W.wall_example1(eps, level)
            p = c.problem
            s = lb.Solver(1, c.N, c.nu, c.dx, c.dt, precision="fx64", stream=stream, boundary=["mirror"])
            with torch.cuda.stream(stream):
                s.set_theta0(torch.from_numpy(p.theta(c.N, c.dx)).cuda(),
                             torch.from_numpy(np.ascontiguousarray(p.grad(c.N, c.dx))).cuda())
                s.step(c.nsteps)
                th, _, u = s.macros(want=("theta", "u"))
            torch.cuda.synchronize()
            T = c.t_end
            rows["theta"].append(float(np.sqrt(np.mean((th.cpu().numpy() - p.theta(c.N, c.dx, T)) ** 2))))
            rows["u"].append(float(np.sqrt(np.mean((u.cpu().numpy()[0] - p.u(c.N, c.dx, T)[0]) ** 2))))
            s.close()
        ex1[str(eps)] = {v: {"rmse": e, "cr": [math.log2(e[i] / e[i + 1]) for i in range(3)],
                             "paper_table1": list(TABLE1[eps][k])} for k, (v, e) in enumerate(rows.items())}
    out["example1"] = {"workload": "1D, walls at x = 0 and 1, u(x,0) = sin(pi x), t = 2, dx = 1/40/2^l, "
                                   "dt = 1/100/4^l, fx64", "by_eps": ex1}
    return out


def run_4d(local, peaks):
    """The paper's Example 4 (D4Q33, periodic [-1,1]^4) at its finest printed
    level: dx = 1/25 (50^4 nodes), dt = 1/250, t = 1 (250 steps), eps = 0.08.
    Sweep throughput per precision, and the closed-node RMSE of the FX64 run
    beside the values the paper prints in Table 4's last column."""
    import torch
    from paper_2309_02825_gb300 import lb
    torch.cuda.set_device(local)
    eps, dx, dt, steps = 0.08, 1.0 / 25, 1.0 / 250, 250
    nu = eps * dx * dx / dt
    N = (50,) * 4
    prob = W.ProductSineProblem(4, nu, (1, 2, 3, 4), 2.0, 2.0, origin=-1.0)
    stream = torch.cuda.Stream()
    th0 = torch.from_numpy(prob.theta(N, dx)).cuda()
    g0 = torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda()
    nodes = 50 ** 4
    out = {"workload": "4D D4Q33 periodic 50^4 (paper Example 4, dx=1/25, dt=1/250, eps=0.08, t=1)"}
    for prec in ("fx64", "fp64", "fp32s"):
        s = lb.Solver(4, N, nu, dx, dt, precision=prec, theta_ref=2.0, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            s.set_theta0(th0, g0)
            s.step(5)
            e0.record(stream)
            s.step(20)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        elem = 4 if prec == "fp32s" else 8
        gbs = 2 * 33 * elem * nodes / (ms / 1e3) / 1e9
        entry = {"sweep_ms": ms, "mlups": nodes / (ms / 1e3) / 1e6, "bytes_per_lu": 2 * 33 * elem,
                 "hbm_frac": gbs / peaks["hbm_gbs"], "traffic": profile_traffic("sweep_d4q33_%s_50" % prec)}
        if prec == "fx64":
            with torch.cuda.stream(stream):
                s.set_theta0(th0, g0)
                s.step(steps)
                th, _, u = s.macros(want=("theta", "u"))
            torch.cuda.synchronize()
            closed = lambda a: np.pad(a, [(0, 1)] * a.ndim, mode="wrap")
            rm = lambda a, b: float(np.sqrt(np.mean((closed(a) - closed(b)) ** 2)))
            T = steps * dt
            the, ue = prob.theta(N, dx, T), prob.u(N, dx, T)
            thh, uh = th.cpu().numpy(), u.cpu().numpy()
            entry["rmse_closed_nodes"] = {"theta": rm(thh, the),
                                          **{"u_x%d" % (a + 1): rm(uh[a], ue[a]) for a in range(4)}}
            entry["paper_table4_last_column"] = {"theta": 8.5486e-9, "u_x1": 1.5000e-9, "u_x2": 2.9646e-9,
                                                 "u_x3": 4.2069e-9, "u_x4": 4.5931e-9}
        s.close()
        out[prec] = entry
    return out


def run_profile_batch(local, spec):
    """Minimal, repeatable command for ncu: the first COUNT instances of the
    batched workload (PREC, default FP32s), STEPS steps; with K,TILE,THREADS
    appended, blocked launches of K steps, else the flat one-launch-per-step
    schedule with the block size the autotuner picks for that precision."""
    import torch
    from paper_2309_02825_gb300 import lb
    torch.cuda.set_device(local)
    parts = spec.split(",")
    count, steps = int(parts[0]), int(parts[1])
    prec = parts[2] if len(parts) > 2 else "fp32s"
    cases = W.batched_2d(512, nsteps=2000)[:count]
    th0 = np.concatenate([c.problem.theta(c.N, c.dx).ravel() for c in cases])
    g0 = np.concatenate([np.ascontiguousarray(c.problem.grad(c.N, c.dx)).ravel() for c in cases])
    kw = {"theta_ref": [1.5] * len(cases)} if prec == "fp32s" else {}
    b = lb.Batch([c.N for c in cases], [c.nu for c in cases], [c.dx for c in cases], [c.dt for c in cases],
                 precision=prec, **kw)
    if len(parts) > 5:
        b.set_blocking(int(parts[3]), int(parts[4]), int(parts[5]), False)
    else:
        b.set_schedule(1e18, 64 if prec == "fx64" else 128, False)
    b.set_theta0(torch.from_numpy(th0).cuda(), torch.from_numpy(g0).cuda())
    b.step(steps)
    torch.cuda.synchronize()
    b.close()
    print(json.dumps({"profile_batch": spec, "ok": True}))


def run_profile_adjoint(local, spec):
    """Minimal, repeatable command for ncu: the adjoint workload's forward
    with checkpoints, seed and T reverse steps at N^2 (PREC storage)."""
    import torch
    from paper_2309_02825_gb300 import lb
    torch.cuda.set_device(local)
    prec, n, T = spec.split(",")
    n, T = int(n), int(T)
    case = W.adjoint_2d(n, T)
    N = case.N
    th0 = torch.from_numpy(case.problem.theta(N, case.dx)).cuda()
    ut = torch.from_numpy(np.ascontiguousarray(case.extra["target"].u(N, case.dx, T * case.dt))).cuda()
    s = lb.Solver(2, N, case.nu, case.dx, case.dt, precision=prec)
    a = lb.Adjoint(s, T, checkpoint=0, want_nu=True)
    u = a.forward(th0)
    a.seed(u - ut)
    a.step(T)
    a.result()
    torch.cuda.synchronize()
    a.close()
    s.close()
    print(json.dumps({"profile_adjoint": spec, "ok": True}))


def run_profile_sweep(local, spec, blocking=None):
    """Minimal, repeatable command for ncu: init + STEPS sweeps of one grid,
    then one recovery, one state sum and the error norms."""
    import torch
    from paper_2309_02825_gb300 import lb
    torch.cuda.set_device(local)
    d, prec, n, steps = spec.split(",")
    d, n, steps = int(d), int(n), int(steps)
    case = {1: W.sine_1d, 2: W.sine_2d, 3: W.fourier_3d}[d](n) if d <= 3 else None
    if case is None:
        dx, dt = 2.0 / n, (2.0 / n) ** 2 / 0.16
        nu = 0.08 * dx * dx / dt
        prob, N = W.ProductSineProblem(4, nu, (1, 2, 3, 4), 2.0, 2.0, origin=-1.0), (n,) * 4
    else:
        prob, N, nu, dx, dt = case.problem, case.N, case.nu, case.dx, case.dt
    s = lb.Solver(d, N, nu, dx, dt, precision=prec, theta_ref=1.5)
    blk = [int(v) for v in blocking.split(",")] if blocking else None
    if blk:
        s.set_blocking(*blk)
    s.set_theta0(torch.from_numpy(prob.theta(N, dx)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx))).cuda())
    for _ in range(steps // blk[0] if blk else steps):
        s.step(blk[0] if blk else 1)
    th, _, u = s.macros(want=("theta", "u"))
    s.sum_theta()
    T = steps * dt
    s.reduce(th, u, torch.from_numpy(prob.theta(N, dx, T)).cuda(),
             torch.from_numpy(np.ascontiguousarray(prob.u(N, dx, T))).cuda())
    torch.cuda.synchronize()
    s.close()
    print(json.dumps({"profile_sweep": spec, "ok": True}))


def run_accuracy(local, precisions=("fp64", "fx64", "fp32s")):
    """Error against the exact solution per grid size and precision, run to
    each family's end time; CR = log2 of successive RMSE ratios."""
    import torch
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    table = {}
    fams = [("1d_sine", W.sine_1d, (16, 32, 64, 128), 2.0), ("2d_sine", W.sine_2d, (64, 128, 256, 512, 1024, 2048, 4096), 2.0),
            ("3d_fourier", W.fourier_3d, (32, 64, 128, 256), 1.5)]
    for name, fam, Ns, tref in fams:
        for prec in precisions:
            rows, prev = [], None
            for N in Ns:
                case = fam(N)
                t0 = time.perf_counter()
                e = _run_case(case, prec, tref, stream)
                e["N"], e["steps"], e["seconds"] = N, case.nsteps, time.perf_counter() - t0
                if prev:
                    e["CR_u"] = math.log2(prev["u_rmse"] / e["u_rmse"])
                    e["CR_theta"] = math.log2(prev["theta_rmse"] / e["theta_rmse"])
                rows.append(e)
                prev = e
            table["%s_%s" % (name, prec)] = rows
    return table


# ---------------------------------------------------------------------------
# The oracle (CPU baseline / reference arm).
# ---------------------------------------------------------------------------

def time_oracle(N, sweeps, threads):
    import oracle as O
    O.set_threads(threads)
    case = W.sine_2d(N)
    m = O.Model(case.d, case.N, case.nu, case.dx, case.dt)
    f = m.initialize(case.problem.theta(case.N, case.dx), case.problem.grad(case.N, case.dx))
    t0 = time.perf_counter()
    f = m.run(f, sweeps)
    el = time.perf_counter() - t0
    return case.nodes * sweeps / el / 1e6, el, O.threads()


def cpu_baseline(args):
    """The FP64 oracle (OpenMP over nodes; bit-identical for any thread count)
    on every host core, and on one core, each on a bounded sample of the
    benchmark's sweeps (about 10 s of CPU work each)."""
    cores = os.cpu_count() or 1
    # one Grace core: about 1.5 s per 4096^2 sweep; all cores: about 10x faster
    s1 = max(8, int(round(8 * (4096.0 / max(args.N, 1)) ** 2)))
    v1, el1, _ = time_oracle(args.N, s1, 1)
    sn = max(8, int(round(10.0 / max(el1 / s1 / min(cores, 12), 1e-6))))
    vn, eln, used = time_oracle(args.N, sn, cores)
    return {"value": vn, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "%d sweeps of the %d^2 D2Q9 FP64 oracle (%.1f s, %d threads)" % (sn, args.N, eln, used),
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": "%d sweeps of the %d^2 D2Q9 FP64 oracle (%.1f s, 1 thread)" % (s1, args.N, el1)}}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, one bounded step per
    benchmark step (initialisation + 1 sweep + recovery of the 2D sine
    workload), on every host core (OpenMP over nodes); rank 0 only."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import oracle as O
    O.set_threads(os.cpu_count() or 1)
    cores = O.threads()
    case = W.sine_2d(args.N)
    th0 = case.problem.theta(case.N, case.dx)
    g0 = case.problem.grad(case.N, case.dx)
    m = O.Model(case.d, case.N, case.nu, case.dx, case.dt)

    def one():
        f = m.initialize(th0, g0)
        f = m.run(f, 1)
        m.recover(f)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    value = case.nodes * args.steps / el / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "2D D2Q9 periodic %d^2 sine, nu=0.02, eps=0.2048; reference step = oracle "
                   "initialisation + 1 sweep + recovery" % args.N, "precision": "fp64",
                   "l2_flush": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d steps of (init + 1 sweep + recovery) at %d^2, %d threads" % (
                             args.steps, args.N, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    world, rank, local = dist_setup(args)
    if args.profile_batch:
        run_profile_batch(local, args.profile_batch)
        return 0
    if args.profile_adjoint:
        run_profile_adjoint(local, args.profile_adjoint)
        return 0
    if args.profile_sweep:
        run_profile_sweep(local, args.profile_sweep, args.blocking)
        return 0
    if args.accuracy:
        if rank == 0:
            print(json.dumps({"accuracy": run_accuracy(local, tuple(args.accuracy_precisions.split(",")))}))
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.slab:
        res = run_slab(args, world, rank, local, 100 * args.steps, 10 * args.warmup)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": res["mlups"], "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_sweep"] * 100,
                              "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int64",
                              "data": "synthetic",
                              "config": {"workload": "2D D2Q9 periodic %d^2 sine, FX64, one grid cut into %d slabs "
                                                     "(step = 100 sweeps, each after a ghost-layer exchange)"
                                                     % (args.N, world), "parallelism": "slab%d" % world},
                              "slab": res}))
        if world > 1:
            dist.destroy_process_group()
        return 0
    peaks = load_peaks()
    main_res = run_ours(args, args.precision, world, rank, local, peaks, not args.no_e2e, True)
    per_step = None
    if main_res["blocking"]["steps_per_launch"]:
        # the same step with one sweep per launch (the HBM-bound sweep)
        v = run_ours(args, args.precision, world, rank, local, peaks, False, False, blocking=False)
        per_step = {"value": v["value"], "unit": UNIT, "sweep_ms": v["sweep_ms"], "roofline": v["roofline"]}
    variants = []
    if not args.no_variant:
        for other in ("fx64", "fp64", "fp32s"):
            if other == args.precision:
                continue
            v = run_ours(args, other, world, rank, local, peaks, False, False)
            entry = {"precision": other, "value": v["value"], "unit": UNIT, "roofline": v["roofline"],
                     "error": v["error"], "sweep_ms": v["sweep_ms"], "blocking": v["blocking"]}
            if "roofline_fp64_pipe" in v:
                entry["roofline_fp64_pipe"] = v["roofline_fp64_pipe"]
            if other == "fp64":
                entry["note"] = ("native FP64 arithmetic, bound by the FP64 pipe (1/64 of the FP32 rate on this part); "
                                 "the FP64-accurate result at the HBM rate and beyond is the 64-bit fixed-point line")
            variants.append(entry)
    batched = None
    if not args.no_batched:
        batched = run_batched(local)
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(local, "fp64")
        for prec in ("fx64", "fp32s"):
            a = run_adjoint(local, prec)
            adjoint[prec] = {k: a[k] for k in ("forward_with_checkpoints_s", "reverse_s", "plain_sweep_us",
                                               "reverse_step_us", "adjoint_step_cost_vs_forward_step",
                                               "gradient_total_cost_vs_forward", "loss", "dL_dnu",
                                               "fd_rel_err_theta0_dirs", "fd_rel_err_nu")}
            adjoint[prec]["dL_dnu_rel_diff_vs_fp64"] = abs(a["dL_dnu"] / adjoint["dL_dnu"] - 1.0)
    sweeps3d = None
    if not args.no_3d:
        sweeps3d = run_3d(local, peaks)
    sweeps4d = None
    if not args.no_4d:
        sweeps4d = run_4d(local, peaks)
    walls = None
    if not args.no_walls:
        walls = run_walls(local, peaks)
    slab_one = None
    if world == 1 and not args.no_walls:
        # the slab path's exchange on one GPU: one part whose buffers wrap onto itself
        slab_one = run_slab(args, 1, 0, local, 200, 20)
    base = None
    if rank == 0 and not args.no_cpu_baseline:
        base = cpu_baseline(args)
    if rank == 0:
        line = {
            "metric": METRIC, "value": main_res["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main_res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32s": "f32", "fx64": "int64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "2D D2Q9 periodic %d^2 sine, nu=0.02, eps=0.2048; step = init + %d fused "
                       "sweeps + recovery + sum theta + error norms" % (args.N, args.sweeps),
                       "precision": args.precision, "sweeps_per_step": args.sweeps,
                       "l2_flush": "inputs larger than L2 (state %.1f GB)" % (
                           2 * 9 * (4 if args.precision == "fp32s" else 8) * args.N ** 2 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": main_res["roofline"],
            "cpu_baseline": base,
            "e2e": main_res.get("e2e"),
            "gpu_launches": main_res["gpu_launches"] * world,
            "clocks": main_res["clocks"],
            "error": main_res["error"],
            "sweep_ms": main_res["sweep_ms"],
        }
        line["blocking"] = main_res["blocking"]
        if per_step:
            line["one_sweep_per_launch"] = per_step
        if "roofline_fp64_pipe" in main_res:
            line["roofline_fp64_pipe"] = main_res["roofline_fp64_pipe"]
        if variants:
            line["variants"] = variants
        if batched:
            line["batched"] = batched
        if adjoint:
            line["adjoint"] = adjoint
        if sweeps3d:
            line["sweeps_3d"] = sweeps3d
        if sweeps4d:
            line["sweeps_4d"] = sweeps4d
        if walls:
            line["walls"] = walls
        if slab_one:
            line["slab_one_part"] = slab_one
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
