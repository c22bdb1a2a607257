// C-ABI of the solver (declared in include/lb.h): argument checks, device
// memory, parameters, and the order of kernel launches.  No arithmetic of
// the method runs on the host beyond the scalar relaxation set.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "lb_internal.cuh"

namespace {

thread_local std::string g_create_err;

lb_status fail(lb_ctx *c, lb_status s, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_create_err = msg;
    return s;
}

lb_status cuda_fail(lb_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(c, LB_ENOMEM, m);
    return fail(c, LB_ECUDA, m);
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

void free_ctx(lb_ctx *c)
{
    if (!c) return;
    lbk::blocked_release(c);
    for (auto &g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->scratch);
    cudaFree(c->dout);
    cudaFree(c->dflag);
    cudaFree(c->gradtmp);
    delete c;
}

// Make the calling thread's current device the context's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(const lb_ctx *c)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != c->device) cudaSetDevice(c->device);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr int64_t kGraphSteps = 32;  // sweeps per recorded graph (even: parity unchanged)

// Record kGraphSteps sweeps starting from buffer `from` on a private stream.
cudaError_t record_sweeps(lb_ctx *c, int from)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaStream_t user = c->stream;
    c->stream = cs;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int p = from;
        for (int64_t k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
            e = lbk::launch_sweep(c, c->f[p], c->f[p ^ 1]);
            p ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[from], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return e;
}

// Read back and clear the recovery and range flags (ctx->dflag[1..2]) after
// the work enqueued so far; synchronises the stream.  A staging timeout or a
// fixed-point range overflow leaves the context uninitialised: the state (or
// a staging tile) may be corrupt, so lb_step and lb_macros refuse to run
// until lb_set_theta0 or lb_load_state sets a state again.
lb_status read_flags(lb_ctx *c, const char *who)
{
    int fl[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(fl, c->dflag + lbk::kFlagRecover, sizeof fl, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dflag + lbk::kFlagRecover, 0, sizeof fl, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, who);
    const std::string w(who);
    if (fl[0] & 4) {
        c->initialized = false;
        return fail(c, LB_ETIMEOUT, w + ": a shared-memory staging wait of the recovery timed out; set the state "
                                        "again (lb_set_theta0 or lb_load_state)");
    }
    if (fl[1]) {
        c->initialized = false;
        return fail(c, LB_EINVAL, w + ": a fixed-point distribution reached |f| >= 2^61 (the run is unstable: an "
                                      "FP64 run would overflow); set the state again");
    }
    if (fl[0]) return fail(c, LB_ENONPOS, w + ": theta <= 0 or non-finite at some node");
    return LB_OK;
}

constexpr int64_t kTbGraphLaunches = 16;  // blocked launches per recorded graph (even)

// Record kTbGraphLaunches blocked launches of tb_k steps starting from buffer `from`.
cudaError_t record_blocked(lb_ctx *c, int from)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int p = from;
        for (int64_t k = 0; k < kTbGraphLaunches && e == cudaSuccess; ++k) {
            e = lbk::blocked_launch(c, c->f[p], c->f[p ^ 1], c->tb_k, cs);
            p ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->tb_graph[from], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return e;
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return true;
    return cap != cudaStreamCaptureStatusNone;
}

}  // namespace

namespace lbk {

bool derive_params(lb_ctx &c, const lb_relax *rs)
{
    const int d = c.d;
    const bool paper = !rs || rs->paper_set;
    c.paper = paper;
    if (paper) {
        const double a = 6.0 * c.eps + 1.0;
        c.s1 = 2.0 / a;
        c.s2x = 24.0 * c.eps / (a * a);
        if (d == 1) {
            c.s22 = 1.0;
            c.w1 = 1.0 / 6.0;
            c.wd = 0.0;
        } else {
            c.s22 = 4.0 / (6.0 * c.eps + 3.0);
            c.w1 = 1.0 / 6.0 - (d - 1) * c.eps / 3.0;
            c.wd = c.eps / 6.0;
        }
    } else {
        c.s1 = rs->s1;
        c.s2x = rs->s2x;
        c.s22 = (d > 1) ? rs->s22 : 1.0;
        c.w1 = rs->w1;
        c.wd = (d > 1) ? rs->wd : 0.0;
    }
    c.theta_ref = rs ? rs->theta_ref : 0.0;
    const bool rates_ok = c.s1 > 0 && c.s1 < 2 && c.s2x > 0 && c.s2x < 2 && (d == 1 || (c.s22 > 0 && c.s22 < 2));
    if (!rates_ok || !isfinite(c.w1) || !isfinite(c.wd) || !isfinite(c.theta_ref)) return false;
    // Eq. (d1-3-weight) and c_s^2 = [2 w1 + 4(d-1) wd] c^2.
    c.w0 = 1.0 - 2.0 * d * c.w1 - 2.0 * d * (d - 1) * c.wd;
    c.sigma = 2.0 * c.w1 + 4.0 * (d - 1) * c.wd;
    c.cs2 = c.sigma * c.c * c.c;
    return true;
}

}  // namespace lbk

extern "C" {

lb_status lb_create(int d, const int64_t *N, double nu, double dx, double dt, const lb_relax *rs, int precision,
                    void *stream, lb_ctx **out)
{
    lbk::NvtxRange nvtx_range("lb_create");
    if (!out) return fail(nullptr, LB_EINVAL, "lb_create: out is NULL");
    *out = nullptr;
    if (d < 1 || d > 4) return fail(nullptr, LB_EINVAL, "lb_create: d must be 1, 2, 3 or 4");
    if (!N) return fail(nullptr, LB_EINVAL, "lb_create: N is NULL");
    if (!finite_pos(nu) || !finite_pos(dx) || !finite_pos(dt))
        return fail(nullptr, LB_EINVAL, "lb_create: nu, dx and dt must be finite and > 0");
    if (precision != LB_FP64 && precision != LB_FP32_SHIFTED && precision != LB_FX64)
        return fail(nullptr, LB_EINVAL, "lb_create: unknown precision");
    int64_t nodes = 1;
    for (int a = 0; a < d; ++a) {
        if (N[a] < 1 || N[a] > (1 << 24)) return fail(nullptr, LB_EINVAL, "lb_create: each N must be in [1, 2^24]");
        nodes *= N[a];
        if (nodes > (int64_t(1) << 31)) return fail(nullptr, LB_EINVAL, "lb_create: more than 2^31 nodes");
    }

    lb_ctx *c = new (std::nothrow) lb_ctx();
    if (!c) return fail(nullptr, LB_ENOMEM, "lb_create: host allocation failed");
    c->d = d;
    c->q = 1 + 2 * d * d;
    for (int a = 0; a < 4; ++a) c->N[a] = (a < d) ? N[a] : 1;
    c->nodes = nodes;
    c->precision = precision;
    c->nu = nu;
    c->dx = dx;
    c->dt = dt;
    c->c = dx / dt;
    c->eps = nu * dt / (dx * dx);
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);

    if (!lbk::derive_params(*c, rs)) {
        free_ctx(c);
        return fail(nullptr, LB_EINVAL, "lb_create: relaxation rates must lie in (0, 2) and weights be finite");
    }
    if (precision == LB_FX64 && !lbk::fx_constants_ok(*c)) {
        free_ctx(c);
        return fail(nullptr, LB_EINVAL, "lb_create: a fixed-point collision constant leaves (-1, 1) (weights too large "
                                        "for LB_FX64; use LB_FP64)");
    }

    // Layout.
    const int V = (precision == LB_FP32_SHIFTED) ? lbk::Vec<float>::V : lbk::Vec<double>::V;
    c->elem = (precision == LB_FP32_SHIFTED) ? 4 : 8;
    const int W = lbk::lane_width(c->d, c->elem, precision == LB_FP64);
    c->geom = lbk::make_geom(c->N[0], c->N[1], c->N[2], c->N[3], V, W);
    const lbk::Geom &g = c->geom;

    const size_t fbytes = ((size_t)c->q * (size_t)g.slab + lbk::kSlackElems) * c->elem;
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        e = cudaMalloc(&c->f[b], fbytes);
        if (e != cudaSuccess) {
            free_ctx(c);
            return cuda_fail(nullptr, e, "lb_create: state allocation");
        }
        e = cudaMemsetAsync(c->f[b], 0, fbytes, c->stream);
        if (e != cudaSuccess) {
            free_ctx(c);
            return cuda_fail(nullptr, e, "lb_create: memset");
        }
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->scratch_blocks = (sms > 0 ? sms : 148) * 4;
    if ((e = cudaMalloc(&c->scratch, sizeof(double) * lbk::kRedSlots * c->scratch_blocks)) != cudaSuccess ||
        (e = cudaMalloc(&c->dout, sizeof(double) * 64)) != cudaSuccess ||
        (e = cudaMalloc(&c->dflag, sizeof(int) * 4)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->dflag, 0, sizeof(int) * 4, c->stream)) != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(nullptr, e, "lb_create: scratch allocation");
    }
    *out = c;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx *c)
{
    lbk::NvtxRange nvtx_range("lb_destroy");
    if (!c) return LB_OK;
    DeviceGuard dg(c);
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return LB_OK;
}

lb_status lb_get_params(const lb_ctx *c, double *out)
{
    if (!c || !out) return LB_EINVAL;
    const double v[15] = {c->eps, c->c,  c->cs2, c->s1, c->s2x, c->s22,       c->w0,       c->w1,
                          c->wd,  c->nu, c->dx,  c->dt, (double)c->q, c->theta_ref, (double)c->fx_bits};
    memcpy(out, v, sizeof v);
    return LB_OK;
}

lb_status lb_set_boundary(lb_ctx *c, const int *kind)
{
    lbk::NvtxRange nvtx_range("lb_set_boundary");
    if (!c) return LB_EINVAL;
    if (!kind) return fail(c, LB_EINVAL, "lb_set_boundary: kind is NULL");
    unsigned mask = 0;
    for (int a = 0; a < c->d; ++a) {
        if (kind[a] != LB_PERIODIC && kind[a] != LB_MIRROR)
            return fail(c, LB_EINVAL, "lb_set_boundary: kind must be LB_PERIODIC or LB_MIRROR");
        if (kind[a] == LB_MIRROR) {
            if (c->N[a] < 3) return fail(c, LB_EINVAL, "lb_set_boundary: a mirror axis needs at least 3 nodes");
            mask |= 1u << a;
        }
    }
    DeviceGuard dg(c);
    // recorded sweeps hold the old geometry; drain the stream before dropping them
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_set_boundary");
    for (auto &g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    c->geom.mirror = mask;
    c->initialized = false;  // the stored state follows the old walls: initialise again
    if (mask) lbk::blocked_release(c);  // blocked sweeps are periodic only
    ++c->gen;
    return LB_OK;
}

lb_status lb_set_viscosity(lb_ctx *c, double nu)
{
    lbk::NvtxRange nvtx_range("lb_set_viscosity");
    if (!c) return LB_EINVAL;
    if (!finite_pos(nu)) return fail(c, LB_EINVAL, "lb_set_viscosity: nu must be finite and > 0");
    lb_ctx trial;
    trial.d = c->d;
    trial.dx = c->dx;
    trial.dt = c->dt;
    trial.c = c->c;
    trial.nu = nu;
    trial.eps = nu * c->dt / (c->dx * c->dx);
    const lb_relax rs = {c->paper ? 1 : 0, c->s1, c->s2x, c->s22, c->w1, c->wd, c->theta_ref};
    if (!lbk::derive_params(trial, &rs))
        return fail(c, LB_EINVAL, "lb_set_viscosity: the relaxation set leaves (0, 2) at this nu");
    if (c->precision == LB_FX64 && !lbk::fx_constants_ok(trial))
        return fail(c, LB_EINVAL, "lb_set_viscosity: a fixed-point collision constant leaves (-1, 1) at this nu");
    DeviceGuard dg(c);
    // recorded sweeps carry the old collision constants; drain the stream before dropping them
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_set_viscosity");
    for (auto &g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    c->nu = nu;
    c->eps = trial.eps;
    c->s1 = trial.s1;
    c->s2x = trial.s2x;
    c->s22 = trial.s22;
    c->w0 = trial.w0;
    c->w1 = trial.w1;
    c->wd = trial.wd;
    c->sigma = trial.sigma;
    c->cs2 = trial.cs2;
    ++c->gen;
    if (c->tb_k > 0) {  // the blocked descriptor carries the collision constants
        bool fits = true;
        if ((e = lbk::blocked_setup(c, c->tb_k, c->tb_tile, c->tb_threads, &fits)) != cudaSuccess)
            return cuda_fail(c, e, "lb_set_viscosity: blocked sweeps");
    }
    return LB_OK;
}

lb_status lb_set_blocking(lb_ctx *c, int steps_per_launch, int tile, int threads)
{
    lbk::NvtxRange nvtx_range("lb_set_blocking");
    if (!c) return LB_EINVAL;
    if (steps_per_launch < 0 || steps_per_launch > 64 ||
        (steps_per_launch > 0 && (tile < 1 || tile > 4096 || !(threads == 256 || threads == 512 || threads == 1024))))
        return fail(c, LB_EINVAL, "lb_set_blocking: steps per launch in 0..64, tile in 1..4096, threads 256, 512 or 1024");
    if (steps_per_launch > 0 && (c->d != 2 || c->geom.mirror))
        return fail(c, LB_EINVAL, "lb_set_blocking: blocked sweeps are built for periodic 2D grids");
    DeviceGuard dg(c);
    cudaError_t e = cudaStreamSynchronize(c->stream);  // tables and graphs may be in use
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_set_blocking");
    bool fits = true;
    if ((e = lbk::blocked_setup(c, steps_per_launch, tile, threads, &fits)) != cudaSuccess)
        return cuda_fail(c, e, "lb_set_blocking");
    if (!fits) return fail(c, LB_EINVAL, "lb_set_blocking: tile plus halo exceeds the shared memory per block");
    return LB_OK;
}

lb_status lb_get_blocking(const lb_ctx *c, int *info)
{
    if (!c || !info) return LB_EINVAL;
    info[0] = c->tb_k;
    info[1] = c->tb_tile;
    info[2] = c->tb_threads;
    info[3] = c->tb_ntiles;
    return LB_OK;
}

lb_status lb_autotune(lb_ctx *c, int trial_steps, double *choice)
{
    lbk::NvtxRange nvtx_range("lb_autotune");
    if (!c || trial_steps < 2) return LB_EINVAL;
    if (c->d != 2 || c->geom.mirror) {  // one sweep per launch is the only schedule here
        if (choice) {
            choice[0] = 0;
            choice[1] = choice[2] = choice[3] = 0;
        }
        return LB_OK;
    }
    DeviceGuard dg(c);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_autotune");
    struct Cand {
        int K, tile, threads;
    };
    std::vector<Cand> cands = {{0, 0, 0}};
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device)) != cudaSuccess)
        return cuda_fail(c, e, "lb_autotune");
    const int node_bytes = 9 * (int)c->elem;
    for (int K : {2, 3, 4, 5, 6, 8, 12})
        for (int per_sm : {1, 2, 3, 4}) {
            const long avail = per_sm == 1 ? optin : optin / per_sm - 1024;
            int edge = (int)floor(sqrt((double)avail / node_bytes));
            while ((long)edge * edge * node_bytes > avail) --edge;
            // the largest square tile for this many blocks per SM, and one 4 nodes smaller (less work per block)
            for (int tile : {edge - 2 * K, edge - 2 * K - 4}) {
                if (tile < 8) continue;
                for (int th : {256, 512, 1024}) cands.push_back({K, tile, th});
            }
        }
    const bool was_init = c->initialized;
    c->initialized = true;  // the trials step whatever the buffers hold
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(c, LB_ECUDA, "lb_autotune: events");
    double best = 1e300;
    Cand win = cands[0];
    lb_status st = LB_OK;
    for (const Cand &cd : cands) {
        bool fits = true;
        if ((e = lbk::blocked_setup(c, cd.K, cd.tile, cd.threads, &fits)) != cudaSuccess) {
            st = cuda_fail(c, e, "lb_autotune");
            break;
        }
        if (!fits) continue;
        const int64_t n = cd.K ? (trial_steps + cd.K - 1) / cd.K * cd.K : trial_steps;
        if ((st = lb_step(c, n)) != LB_OK) break;  // warm-up
        if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) {
            st = cuda_fail(c, e, "lb_autotune");
            break;
        }
        if ((st = lb_step(c, n)) != LB_OK) break;
        float ms = 0.f;
        if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
            st = cuda_fail(c, e, "lb_autotune");
            break;
        }
        if (ms / n < best) {
            best = ms / n;
            win = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    c->initialized = false;  // the trials overwrote the state: set it again
    c->step = 0;
    (void)was_init;
    if (st != LB_OK) return st;
    bool fits = true;
    if ((e = lbk::blocked_setup(c, win.K, win.tile, win.threads, &fits)) != cudaSuccess)
        return cuda_fail(c, e, "lb_autotune");
    if (choice) {
        choice[0] = win.K;
        choice[1] = win.tile;
        choice[2] = win.threads;
        choice[3] = 1e3 * best;
    }
    return LB_OK;
}

lb_status lb_get_boundary(const lb_ctx *c, int *kind)
{
    if (!c || !kind) return LB_EINVAL;
    for (int a = 0; a < c->d; ++a) kind[a] = ((c->geom.mirror >> a) & 1u) ? LB_MIRROR : LB_PERIODIC;
    return LB_OK;
}

lb_status lb_set_theta0(lb_ctx *c, const double *theta0, const double *grad)
{
    lbk::NvtxRange nvtx_range("lb_set_theta0");
    if (!c) return LB_EINVAL;
    if (!theta0) return fail(c, LB_EINVAL, "lb_set_theta0: theta0 is NULL");
    DeviceGuard dg(c);
    cudaError_t e;
    c->initialized = false;
    if (!grad) {
        if (!c->gradtmp) {
            e = cudaMalloc(&c->gradtmp, sizeof(double) * c->d * c->nodes);
            if (e != cudaSuccess) return cuda_fail(c, e, "lb_set_theta0: gradient buffer");
        }
        if ((e = lbk::launch_fd4_grad(c, theta0, c->gradtmp)) != cudaSuccess)
            return cuda_fail(c, e, "lb_set_theta0: fd4 launch");
        grad = c->gradtmp;
    }
    if ((e = cudaMemsetAsync(c->dflag, 0, sizeof(int) * 3, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "lb_set_theta0: flag reset");
    if (c->precision == LB_FX64) {
        // Fixed-point scale: max|theta0| * 2^F < 2^59.  Every moment sum is
        // bounded by sum_k |f_k|, which stays near theta for a stable run, so
        // 4 bits of headroom (16 max|theta0|) cover the sums and transients;
        // the initialisation flags any value beyond 4 max|theta0|.
        double mx = 0.0;
        if ((e = lbk::launch_maxabs(c, theta0, c->nodes, c->dout)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&mx, c->dout, sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "lb_set_theta0: max|theta0|");
        if (c->fx_max > 0.0) {  // a slab: the scale of the whole grid (at least this part's maximum)
            if (!isfinite(mx) || mx > c->fx_max)
                return fail(c, LB_EINVAL, "lb_set_theta0: max|theta0| of this part exceeds the grid's maximum");
            mx = c->fx_max;
        }
        if (!(mx > 0.0) || !isfinite(mx)) return fail(c, LB_ENONPOS, "lb_set_theta0: theta0 must be finite and > 0");
        int ex = 0;
        frexp(mx, &ex);  // mx < 2^ex
        c->fx_bits = 59 - ex;
        if (c->fx_bits > 1000 || c->fx_bits < -1000)
            return fail(c, LB_EINVAL, "lb_set_theta0: theta0 magnitude outside the fixed-point range");
    }
    c->cur = 0;
    if ((e = lbk::launch_init(c, theta0, grad, c->dflag)) != cudaSuccess)
        return cuda_fail(c, e, "lb_set_theta0: init launch");
    int flag = 0;
    if ((e = cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "lb_set_theta0");
    if (flag & 2) return fail(c, LB_EINVAL, "lb_set_theta0: initial distributions exceed the fixed-point range");
    if (flag) return fail(c, LB_ENONPOS, "lb_set_theta0: theta0 must be finite and > 0 (and grad finite)");
    c->initialized = true;
    c->step = 0;
    return LB_OK;
}

lb_status lb_step(lb_ctx *c, int64_t nsteps)
{
    lbk::NvtxRange nvtx_range("lb_step");
    if (!c) return LB_EINVAL;
    if (nsteps < 0) return fail(c, LB_EINVAL, "lb_step: nsteps < 0");
    if (!c->initialized) return fail(c, LB_ESTATE, "lb_step: call lb_set_theta0 first");
    DeviceGuard dg(c);
    // Long runs replay recorded 32-sweep graphs (one host call per 32 sweeps);
    // while the caller's stream is being captured the sweeps are launched
    // directly so that they land in the caller's graph.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
    if (c->tb_k > 0) {
        // blocked: launches of tb_k steps (recorded in graphs), then one launch for the remainder
        int64_t launches = nsteps / c->tb_k;
        const int rem = (int)(nsteps % c->tb_k);
        cudaError_t e = cudaSuccess;
        while (cap == cudaStreamCaptureStatusNone && launches >= kTbGraphLaunches) {
            if (!c->tb_graph[c->cur]) e = record_blocked(c, c->cur);
            if (e == cudaSuccess) e = cudaGraphLaunch(c->tb_graph[c->cur], c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "lb_step: blocked graph");
            launches -= kTbGraphLaunches;
            c->step += kTbGraphLaunches * c->tb_k;
        }
        for (; launches > 0; --launches) {
            if ((e = lbk::blocked_launch(c, c->f[c->cur], c->f[c->cur ^ 1], c->tb_k, c->stream)) != cudaSuccess)
                return cuda_fail(c, e, "lb_step: blocked launch");
            c->cur ^= 1;
            c->step += c->tb_k;
        }
        if (rem > 0) {
            if ((e = lbk::blocked_launch(c, c->f[c->cur], c->f[c->cur ^ 1], rem, c->stream)) != cudaSuccess)
                return cuda_fail(c, e, "lb_step: blocked launch");
            c->cur ^= 1;
            c->step += rem;
        }
        return LB_OK;
    }
    while (cap == cudaStreamCaptureStatusNone && nsteps >= kGraphSteps) {
        cudaError_t e = cudaSuccess;
        if (!c->graph[c->cur]) e = record_sweeps(c, c->cur);
        if (e == cudaSuccess) e = cudaGraphLaunch(c->graph[c->cur], c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "lb_step: graph");
        nsteps -= kGraphSteps;
        c->step += kGraphSteps;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaError_t e = lbk::launch_sweep(c, c->f[c->cur], c->f[c->cur ^ 1]);
        if (e != cudaSuccess) return cuda_fail(c, e, "lb_step: sweep launch");
        c->cur ^= 1;
        ++c->step;
    }
    return LB_OK;
}

lb_status lb_get_step(const lb_ctx *c, int64_t *n)
{
    if (!c || !n) return LB_EINVAL;
    *n = c->step;
    return LB_OK;
}

lb_status lb_macros(lb_ctx *c, double *theta, double *grad, double *u)
{
    lbk::NvtxRange nvtx_range("lb_macros");
    if (!c) return LB_EINVAL;
    if (!c->initialized) return fail(c, LB_ESTATE, "lb_macros: call lb_set_theta0 first");
    if (!theta && !grad && !u) return LB_OK;
    DeviceGuard dg(c);
    cudaError_t e = lbk::launch_macros(c, c->f[c->cur], theta, grad, u, c->dflag + lbk::kFlagRecover);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_macros: launch");
    // inside the caller's stream capture nothing can be read back: the flags
    // then wait for lb_check, lb_sum_theta or lb_reduce
    if (capturing(c->stream)) return LB_OK;
    return read_flags(c, "lb_macros");
}

lb_status lb_check(lb_ctx *c)
{
    lbk::NvtxRange nvtx_range("lb_check");
    if (!c) return LB_EINVAL;
    DeviceGuard dg(c);
    return read_flags(c, "lb_check");
}

lb_status lb_sum_theta(lb_ctx *c, double *out)
{
    lbk::NvtxRange nvtx_range("lb_sum_theta");
    if (!c || !out) return LB_EINVAL;
    if (!c->initialized) return fail(c, LB_ESTATE, "lb_sum_theta: call lb_set_theta0 first");
    DeviceGuard dg(c);
    cudaError_t e = lbk::launch_sum_state(c, c->f[c->cur], c->dout);
    double v = 0.0;
    int range = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, c->dout, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&range, c->dflag + lbk::kFlagRange, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dflag + lbk::kFlagRange, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_sum_theta");
    if (range) {
        c->initialized = false;
        return fail(c, LB_EINVAL, "lb_sum_theta: a fixed-point distribution reached |f| >= 2^61 (the run is "
                                  "unstable: an FP64 run would overflow); set the state again");
    }
    if (c->precision == LB_FP32_SHIFTED) {
        // sum of the node weights: N_a per periodic axis, N_a - 1 per mirror axis
        double wn = 1.0;
        for (int a = 0; a < c->d; ++a) wn *= (double)(((c->geom.mirror >> a) & 1u) ? c->N[a] - 1 : c->N[a]);
        v += c->theta_ref * wn;
    }
    *out = v;
    return LB_OK;
}

lb_status lb_reduce(lb_ctx *c, const double *theta, const double *u, const double *ex_theta, const double *ex_u,
                    double *out)
{
    lbk::NvtxRange nvtx_range("lb_reduce");
    if (!c || !out) return LB_EINVAL;
    if (!theta || !ex_theta) return fail(c, LB_EINVAL, "lb_reduce: theta and exact_theta are required");
    if ((u == nullptr) != (ex_u == nullptr)) return fail(c, LB_EINVAL, "lb_reduce: u and exact_u go together");
    DeviceGuard dg(c);
    const int ns = 3 * (c->d + 1) + 1;
    cudaError_t e = lbk::launch_norms(c, theta, u, ex_theta, ex_u, c->dout);
    double raw[lbk::kRedSlots];
    int flag = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(raw, c->dout, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&flag, c->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dflag + 1, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_reduce");
    const double n = (double)c->nodes;
    for (int v = 0; v <= c->d; ++v) {
        const double se = raw[3 * v], mx = raw[3 * v + 1], sx = raw[3 * v + 2];
        const bool have = (v == 0) || u;
        out[3 * v + 0] = have ? sqrt(se / n) : NAN;
        out[3 * v + 1] = have ? mx : NAN;
        out[3 * v + 2] = have ? (sx > 0 ? sqrt(se / sx) : (se > 0 ? INFINITY : 0.0)) : NAN;
    }
    out[3 * (c->d + 1)] = raw[ns - 1];
    if (flag & 4) {
        c->initialized = false;
        return fail(c, LB_ETIMEOUT, "lb_macros: a shared-memory staging wait timed out");
    }
    if (flag) return fail(c, LB_ENONPOS, "lb_macros saw theta <= 0 or non-finite");
    return LB_OK;
}

lb_status lb_state_layout(const lb_ctx *c, int64_t *pitch, int64_t *slab, int64_t *elem_bytes)
{
    if (!c) return LB_EINVAL;
    if (pitch) *pitch = c->geom.pitch;
    if (slab) *slab = c->geom.slab;
    if (elem_bytes) *elem_bytes = (int64_t)c->elem;
    return LB_OK;
}

lb_status lb_save_state(lb_ctx *c, void *buf)
{
    lbk::NvtxRange nvtx_range("lb_save_state");
    if (!c || !buf) return LB_EINVAL;
    if (!c->initialized) return fail(c, LB_ESTATE, "lb_save_state: nothing to save");
    DeviceGuard dg(c);
    cudaError_t e = cudaMemcpyAsync(buf, c->f[c->cur], (size_t)c->q * c->geom.slab * c->elem,
                                    cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_save_state");
    return LB_OK;
}

lb_status lb_load_state(lb_ctx *c, const void *buf, int64_t step)
{
    lbk::NvtxRange nvtx_range("lb_load_state");
    if (!c || !buf || step < 0) return LB_EINVAL;
    DeviceGuard dg(c);
    cudaError_t e = cudaMemcpyAsync(c->f[c->cur], buf, (size_t)c->q * c->geom.slab * c->elem,
                                    cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dflag + lbk::kFlagRecover, 0, sizeof(int) * 2, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_load_state");
    c->initialized = true;
    c->step = step;
    return LB_OK;
}

const char *lb_last_error(const lb_ctx *c)
{
    if (!c) return g_create_err.c_str();
    return c->err.c_str();
}

}  // extern "C"
