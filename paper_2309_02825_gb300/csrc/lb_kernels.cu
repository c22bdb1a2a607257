// CUDA kernels of the MRT-LB hot path (sm_103a).
//
// Sweep = pull-stream + MRT collision of Eq. (distribution-f), fused, one
// warp per row segment of 32*V nodes (V = 2 doubles or 4 floats per thread,
// one 16-byte vector per population).  Populations with e_x = 0 are plain
// aligned vector loads; e_x = +-1 shifts by one element, done with an
// aligned vector load plus one warp shuffle, and a scalar load only at the
// warp edge and the periodic wrap.  Every store is an aligned vector.
//
// The collision is written in moment space in closed form (no q x q
// product): from theta, J_a = sum e_a f, P_aa = sum e_a^2 f and
// P_ab = sum e_a e_b f the relaxed moments follow from S; third-order
// moments relax to 0 and fourth-order ones to 4 wd theta (rate 1), so they
// are never formed; M^-1 is applied analytically.
#include <math.h>

#include "lb_device.cuh"

namespace lbk {

// ---------------------------------------------------------------------------
// Initialisation, written in P form: P_0(y, i) = f_i(y + e_i, 0) with
// f_i = w_i theta0 - dt [M^-1 S^-1 M Dbar f^eq]_i in closed form.
// ---------------------------------------------------------------------------
template <class L, typename T>
__global__ void init_kernel(T *__restrict__ dst, Geom g, InitK K, const double *__restrict__ theta0,
                            const double *__restrict__ grad, int *__restrict__ flag)
{
    const int64_t nodes = (int64_t)g.N0 * g.rows;
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nodes) return;
    const int x = (int)(node % g.N0);
    const int64_t rw = node / g.N0;
    const int y = (int)(rw % g.N1);
    const int z = (int)((rw / g.N1) % g.N2);
    const int w = (int)(rw / ((int64_t)g.N1 * g.N2));
    {
        const double t0 = theta0[node];
        bool bad = !(t0 > 0.0) || !isfinite(t0);
#pragma unroll
        for (int a = 0; a < L::D; ++a) bad |= !isfinite(grad[a * nodes + node]);
        if (bad) atomicOr(flag, 1);
    }
    T *out = dst + (((int64_t)w * g.N2 + z) * g.N1 + y) * g.pitch + x;
    bool range = false;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::E[i][0], ey = L::E[i][1], ez = L::E[i][2], ew = L::E[i][3];
        const int xs = wrapi(x + ex, g.N0);
        const int ys = wrapi(y + ey, g.N1);
        const int zs = wrapi(z + ez, g.N2);
        const int ws = wrapi(w + ew, g.N3);
        const int64_t src = (((int64_t)ws * g.N2 + zs) * g.N1 + ys) * g.N0 + xs;
        const double th = theta0[src];
        double val;
        constexpr int nz = (ex != 0) + (ey != 0) + (ez != 0) + (ew != 0);
        if constexpr (nz == 0) {
            val = K.w0 * th;
        } else if constexpr (nz == 1) {
            constexpr int a = (ex != 0) ? 0 : ((ey != 0) ? 1 : ((ez != 0) ? 2 : 3));
            constexpr int s = (ex != 0) ? ex : ((ey != 0) ? ey : ((ez != 0) ? ez : ew));
            val = K.w1 * th - (double)s * K.iax * grad[a * nodes + src];
            val -= K.w1 * K.theta_ref;
        } else {
            double edg = 0.0;
            if constexpr (ex != 0) edg += (double)ex * grad[src];
            if constexpr (ey != 0) edg += (double)ey * grad[nodes + src];
            if constexpr (ez != 0) edg += (double)ez * grad[2 * nodes + src];
            if constexpr (ew != 0) edg += (double)ew * grad[3 * nodes + src];
            val = K.wd * th - K.idg * edg;
            val -= K.wd * K.theta_ref;
        }
        if constexpr (nz == 0) val -= K.w0 * K.theta_ref;
        out[(int64_t)i * g.slab] = to_store<T>(val, K.fxscale, range);
    });
    if (range) atomicOr(flag, 2);
}

// Fourth-order central difference of theta along each axis (periodic).
__global__ void fd4_kernel(const double *__restrict__ th, double *__restrict__ grad, int d, int N0, int N1,
                           int N2, int N3, double inv12dx)
{
    const int64_t nodes = (int64_t)N0 * N1 * N2 * N3;
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nodes) return;
    int64_t rest = node;
    const int x = (int)(rest % N0);
    rest /= N0;
    const int y = (int)(rest % N1);
    rest /= N1;
    const int z = (int)(rest % N2);
    const int w = (int)(rest / N2);
    const int n[4] = {N0, N1, N2, N3};
    for (int a = 0; a < d; ++a) {
        double acc = 0.0;
        const int off[4] = {2, 1, -1, -2};
        const double cof[4] = {-1.0, 8.0, -8.0, 1.0};
        for (int k = 0; k < 4; ++k) {
            int c[4] = {x, y, z, w};
            c[a] = ((c[a] + off[k]) % n[a] + n[a]) % n[a];
            acc += cof[k] * th[(((int64_t)c[3] * N2 + c[2]) * N1 + c[1]) * N0 + c[0]];
        }
        grad[a * nodes + node] = acc * inv12dx;
    }
}

// ---------------------------------------------------------------------------
// Deterministic FP64 reductions: per-block partials (warp shuffles, then
// shared memory), then one block folds the partials in a fixed order.
// ---------------------------------------------------------------------------
template <int NS> struct Acc {
    double v[NS];
};

// op[k]: 0 = sum, 1 = max
template <int NS>
__device__ __forceinline__ void block_reduce_store(Acc<NS> &a, const int (&op)[NS], double *dst)
{
    __shared__ double sh[kRedThreads / 32][NS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_xor_sync(0xffffffffu, a.v[k], o);
            a.v[k] = op[k] ? fmax(a.v[k], t) : a.v[k] + t;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k) sh[wid][k] = a.v[k];
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        const int k = threadIdx.x;
        double s = sh[0][k];
        for (int w = 1; w < kRedThreads / 32; ++w) s = op[k] ? fmax(s, sh[w][k]) : s + sh[w][k];
        dst[k] = s;
    }
}

// Sum of the stored state over populations and valid nodes.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) sum_state_kernel(const T *__restrict__ src, Geom g, int q,
                                                                double scale, double *__restrict__ partial)
{
    Acc<1> a{{0.0}};
    const int64_t total = (int64_t)q * g.rows * g.N0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.N0);
        const int64_t rr = t / g.N0;  // population * rows + row
        a.v[0] += (double)src[rr * g.pitch + x] * scale;
    }
    const int op[1] = {0};
    block_reduce_store<1>(a, op, partial + (int64_t)blockIdx.x * kRedSlots);
}

// Error norms: slots 3v+0 sum err^2, 3v+1 max |err|, 3v+2 sum exact^2 for
// v = 0 (theta), 1..d (u); slot 3(d+1) = sum theta.
template <int D>
__global__ void __launch_bounds__(kRedThreads) norms_kernel(const double *__restrict__ th,
                                                            const double *__restrict__ u,
                                                            const double *__restrict__ eth,
                                                            const double *__restrict__ eu, int64_t nodes,
                                                            double *__restrict__ partial)
{
    constexpr int NS = 3 * (D + 1) + 1;
    Acc<NS> a;
#pragma unroll
    for (int k = 0; k < NS; ++k) a.v[k] = 0.0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nodes;
         n += (int64_t)gridDim.x * blockDim.x) {
        const double t = th[n], te = eth[n];
        const double e = t - te;
        a.v[0] += e * e;
        a.v[1] = fmax(a.v[1], fabs(e));
        a.v[2] += te * te;
        a.v[NS - 1] += t;
        if (u) {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double uv = u[c * nodes + n], ue = eu[c * nodes + n];
                const double eu2 = uv - ue;
                a.v[3 * (c + 1) + 0] += eu2 * eu2;
                a.v[3 * (c + 1) + 1] = fmax(a.v[3 * (c + 1) + 1], fabs(eu2));
                a.v[3 * (c + 1) + 2] += ue * ue;
            }
        }
    }
    int op[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) op[k] = (k < NS - 1 && k % 3 == 1) ? 1 : 0;
    block_reduce_store<NS>(a, op, partial + (int64_t)blockIdx.x * kRedSlots);
}

// max |x| over n values.
__global__ void __launch_bounds__(kRedThreads) maxabs_kernel(const double *__restrict__ x, int64_t n,
                                                             double *__restrict__ partial)
{
    Acc<1> a{{0.0}};
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        a.v[0] = fmax(a.v[0], fabs(x[t]));
    const int op[1] = {1};
    block_reduce_store<1>(a, op, partial + (int64_t)blockIdx.x * kRedSlots);
}

// Fold nb partial rows of kRedSlots in a fixed order.  opmask bit k = max.
__global__ void __launch_bounds__(kRedThreads) fold_kernel(const double *__restrict__ partial, int nb, int ns,
                                                           unsigned opmask, double *__restrict__ out)
{
    __shared__ double sh[kRedThreads];
    for (int k = 0; k < ns; ++k) {
        const bool mx = (opmask >> k) & 1u;
        double s = mx ? 0.0 : 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const double v = partial[(int64_t)b * kRedSlots + k];
            s = mx ? fmax(s, v) : s + v;
        }
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = mx ? fmax(sh[threadIdx.x], sh[threadIdx.x + w])
                                                       : sh[threadIdx.x] + sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host-side dispatch.
// ---------------------------------------------------------------------------
template <typename T> Coll<T> make_coll(const lb_ctx &cc)
{
    const lb_ctx *c = &cc;
    const double d = c->d;
    const double s2x = c->s2x, s22 = (c->d > 1) ? c->s22 : 1.0, wd = (c->d > 1) ? c->wd : 0.0;
    Coll<T> k;
    k.k1 = (T)((1.0 - c->s1) / 2.0);
    k.k2 = (T)((1.0 - s2x) / 2.0);
    k.k3 = (T)((1.0 - s22) / 4.0);
    k.c0 = (T)(1.0 - d * s2x * c->sigma + 2.0 * d * (d - 1.0) * wd);
    k.cA = (T)(s2x * c->sigma / 2.0 - 2.0 * (d - 1.0) * wd);
    k.wd = (T)wd;
    return k;
}
template Coll<double> make_coll<double>(const lb_ctx &);
template Coll<float> make_coll<float>(const lb_ctx &);


template <class L, typename T> static cudaError_t sweep_t(lb_ctx *c, const void *src, void *dst)
{
    constexpr int TH = sweep_threads<T>();
    const unsigned nb = (unsigned)((c->geom.nseg + TH / 32 - 1) / (TH / 32));
    sweep_kernel<L, T, Coll<T>><<<nb, TH, 0, c->stream>>>(
        (const T *)src, (T *)dst, c->geom, make_coll<T>(*c));
    return cudaGetLastError();
}

cudaError_t launch_sweep(lb_ctx *c, const void *src, void *dst)
{
    if (c->precision == LB_FX64) return launch_sweep_fx(c, src, dst);
    const bool f64 = c->precision == LB_FP64;
    switch (c->d) {
    case 1: return f64 ? sweep_t<D1Q3, double>(c, src, dst) : sweep_t<D1Q3, float>(c, src, dst);
    case 2: return f64 ? sweep_t<D2Q9, double>(c, src, dst) : sweep_t<D2Q9, float>(c, src, dst);
    case 3: return f64 ? sweep_t<D3Q19, double>(c, src, dst) : sweep_t<D3Q19, float>(c, src, dst);
    default: return f64 ? sweep_t<D4Q33, double>(c, src, dst) : sweep_t<D4Q33, float>(c, src, dst);
    }
}

cudaError_t launch_fd4_grad(const lb_ctx *c, const double *theta0, double *grad)
{
    const int64_t nodes = c->nodes;
    fd4_kernel<<<(unsigned)((nodes + 255) / 256), 256, 0, c->stream>>>(
        theta0, grad, c->d, (int)c->N[0], (int)c->N[1], (int)c->N[2], (int)c->N[3], 1.0 / (12.0 * c->dx));
    return cudaGetLastError();
}

template <class L, typename T>
static cudaError_t init_t(lb_ctx *c, const double *theta0, const double *grad, int *flag)
{
    InitK K;
    const double d = c->d;
    const double wd = (c->d > 1) ? c->wd : 0.0;
    K.w0 = c->w0;
    K.w1 = c->w1;
    K.wd = wd;
    K.iax = 0.5 * c->dx * (c->sigma / c->s1 - 4.0 * (d - 1.0) * wd);
    K.idg = wd * c->dx;
    K.theta_ref = (c->precision == LB_FP32_SHIFTED) ? c->theta_ref : 0.0;
    K.fxscale = ldexp(1.0, c->fx_bits);
    init_kernel<L, T><<<(unsigned)((c->nodes + 255) / 256), 256, 0, c->stream>>>(
        (T *)c->f[c->cur], c->geom, K, theta0, grad, flag);
    return cudaGetLastError();
}

cudaError_t launch_init(lb_ctx *c, const double *theta0, const double *grad, int *flag)
{
    if (c->precision == LB_FX64) {
        switch (c->d) {
        case 1: return init_t<D1Q3, long long>(c, theta0, grad, flag);
        case 2: return init_t<D2Q9, long long>(c, theta0, grad, flag);
        case 3: return init_t<D3Q19, long long>(c, theta0, grad, flag);
        default: return init_t<D4Q33, long long>(c, theta0, grad, flag);
        }
    }
    const bool f64 = c->precision == LB_FP64;
    switch (c->d) {
    case 1: return f64 ? init_t<D1Q3, double>(c, theta0, grad, flag) : init_t<D1Q3, float>(c, theta0, grad, flag);
    case 2: return f64 ? init_t<D2Q9, double>(c, theta0, grad, flag) : init_t<D2Q9, float>(c, theta0, grad, flag);
    case 3: return f64 ? init_t<D3Q19, double>(c, theta0, grad, flag) : init_t<D3Q19, float>(c, theta0, grad, flag);
    default: return f64 ? init_t<D4Q33, double>(c, theta0, grad, flag) : init_t<D4Q33, float>(c, theta0, grad, flag);
    }
}

cudaError_t launch_sum_state(lb_ctx *c, const void *src, double *out_dev)
{
    const int nb = c->scratch_blocks;
    if (c->precision == LB_FP64)
        sum_state_kernel<double><<<nb, kRedThreads, 0, c->stream>>>((const double *)src, c->geom, c->q, 1.0,
                                                                     c->scratch);
    else if (c->precision == LB_FX64)
        sum_state_kernel<long long><<<nb, kRedThreads, 0, c->stream>>>(
            (const long long *)src, c->geom, c->q, ldexp(1.0, -c->fx_bits), c->scratch);
    else
        sum_state_kernel<float><<<nb, kRedThreads, 0, c->stream>>>((const float *)src, c->geom, c->q, 1.0,
                                                                    c->scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_kernel<<<1, kRedThreads, 0, c->stream>>>(c->scratch, nb, 1, 0u, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_maxabs(lb_ctx *c, const double *x, int64_t n, double *out_dev)
{
    const int nb = c->scratch_blocks;
    maxabs_kernel<<<nb, kRedThreads, 0, c->stream>>>(x, n, c->scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_kernel<<<1, kRedThreads, 0, c->stream>>>(c->scratch, nb, 1, 1u, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_norms(lb_ctx *c, const double *th, const double *u, const double *eth, const double *eu,
                         double *out_dev)
{
    const int nb = c->scratch_blocks;
    const int ns = 3 * (c->d + 1) + 1;
    unsigned mask = 0;
    for (int k = 0; k < ns - 1; ++k)
        if (k % 3 == 1) mask |= 1u << k;
    switch (c->d) {
    case 1: norms_kernel<1><<<nb, kRedThreads, 0, c->stream>>>(th, u, eth, eu, c->nodes, c->scratch); break;
    case 2: norms_kernel<2><<<nb, kRedThreads, 0, c->stream>>>(th, u, eth, eu, c->nodes, c->scratch); break;
    case 3: norms_kernel<3><<<nb, kRedThreads, 0, c->stream>>>(th, u, eth, eu, c->nodes, c->scratch); break;
    default: norms_kernel<4><<<nb, kRedThreads, 0, c->stream>>>(th, u, eth, eu, c->nodes, c->scratch); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_kernel<<<1, kRedThreads, 0, c->stream>>>(c->scratch, nb, ns, mask, out_dev);
    return cudaGetLastError();
}

// Norm reduction into caller-provided partial rows (nblocks of kRedSlots)
// and one raw-sum row; used by the allocation-free entry point.
cudaError_t launch_norms_into(int d, int64_t nodes, const double *th, const double *u, const double *eth,
                              const double *eu, double *partials, int nb, double *raw_out, cudaStream_t s)
{
    const int ns = 3 * (d + 1) + 1;
    unsigned mask = 0;
    for (int k = 0; k < ns - 1; ++k)
        if (k % 3 == 1) mask |= 1u << k;
    switch (d) {
    case 1: norms_kernel<1><<<nb, kRedThreads, 0, s>>>(th, u, eth, eu, nodes, partials); break;
    case 2: norms_kernel<2><<<nb, kRedThreads, 0, s>>>(th, u, eth, eu, nodes, partials); break;
    default: norms_kernel<3><<<nb, kRedThreads, 0, s>>>(th, u, eth, eu, nodes, partials); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_kernel<<<1, kRedThreads, 0, s>>>(partials, nb, ns, mask, raw_out);
    return cudaGetLastError();
}

}  // namespace lbk
