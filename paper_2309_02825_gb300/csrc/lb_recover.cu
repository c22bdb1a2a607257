// Macroscopic recovery (Sec. III.C) with TMA-staged halos.
//
// Each block recovers one row segment of kTile nodes.  For every population
// i it copies the source row segment [x0 - H, x0 + kTile + H) (H = one
// 16-byte vector, clipped to the row) from HBM into shared memory with one
// bulk asynchronous copy (cp.async.bulk, completing on an mbarrier), so the
// one-node x-halo that the pull f_i(x) = P_i(x - e_i) needs arrives with
// the tile; only the two periodic wrap nodes of a row (x = 0 pulling from
// N0 - 1, x = N0 - 1 pulling from 0) read a scalar from global memory.
// Then theta = sum f, J = sum e f (exact integer sums for 64-bit fixed
// point), grad theta = -s1 J / (sigma dx) and u = (2 - s1) c J / theta.
// With mirror walls (MIR) a row or population beyond a wall is read from its
// reflection (pop_source), and the wall nodes of x read x = 1 and N0 - 2 of
// the x-reflected population instead of the periodic wrap.
// The mbarrier wait is bounded: on timeout the block records an error flag,
// waits (again bounded) for its own copies and returns.
#include <math.h>
#include <stdint.h>

#include "lb_device.cuh"

namespace lbk {

constexpr int kTile = 256;                          // nodes per block (one per thread)
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s bound on a staging wait

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Non-blocking test of an mbarrier phase.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Poll the phase until it completes or limit_ns of wall time have passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_test_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

template <typename T> struct RecAcc {
    using type = double;
};
template <> struct RecAcc<long long> {
    using type = long long;  // exact integer moment sums
};

// Rows row0 .. row0 + nrow - 1 of the grid (all rows in a plain recovery);
// the outputs hold those rows only, node (row - row0) * N0 + x.
template <class L, typename T, bool MIR>
__global__ void __launch_bounds__(kTile) recover_kernel(const T *__restrict__ src, Geom g, Recov r, double scale,
                                                       double *__restrict__ theta, double *__restrict__ grad,
                                                       double *__restrict__ u, int *__restrict__ flag, int64_t row0,
                                                       int64_t nrow)
{
    constexpr int H = 16 / (int)sizeof(T);  // halo = one 16-byte vector
    constexpr int TW = kTile + 2 * H;        // tile width per population
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    __shared__ __align__(8) unsigned long long bar;

    const int tiles_per_row = (g.N0 + kTile - 1) / kTile;
    const int64_t row = row0 + blockIdx.x / tiles_per_row;
    const int x0 = (int)(blockIdx.x % tiles_per_row) * kTile;
    const RowPos rpos = row_pos<L::D>(g, row);
    // copy window: multiples of H elements, i.e. 16-byte aligned and sized
    const int xs = max(x0 - H, 0);
    const int xe = min(x0 + kTile + H, g.pitch);
    const uint32_t bytes = (uint32_t)((xe - xs) * (int)sizeof(T));
    const uint32_t barp = smem_u32(&bar);

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(barp), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(barp),
                     "r"(bytes * (uint32_t)L::Q)
                     : "memory");
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const PopSrc ps = pop_source<L, i, MIR>(g, rpos);
            const T *gsrc = src + (int64_t)ps.pop * g.slab + ps.row * g.pitch + xs;
            const uint32_t dst = smem_u32(tile + i * TW + (xs - x0 + H));
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                "l"(gsrc), "r"(bytes), "r"(barp)
                : "memory");
        });
    }
    if (!mbar_wait_bounded(barp, 0)) {
        if (threadIdx.x == 0) atomicOr(flag, 4);
        // Give this block's copies a second bounded interval to land before its
        // shared memory goes away.  If that also runs out the block returns with
        // copies possibly still in flight; the host treats flag bit 2 as fatal
        // for the context's state (lb_macros returns LB_ETIMEOUT and the context
        // needs a new state before it launches again).
        mbar_wait_bounded(barp, 0);
        return;
    }

    const int x = x0 + (int)threadIdx.x;
    if (x >= g.N0) return;
    T vals[L::Q];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::E[i][0];
        const int sx = x - ex;
        if (sx >= 0 && sx < g.N0) {
            vals[i] = tile[i * TW + (sx - x0 + H)];
        } else {  // across the row end: a scalar from the other end, or the x-reflection
            const PopSrc ps = pop_source<L, i, MIR>(g, rpos);
            if (MIR && (g.mirror & 1u))
                vals[i] = src[(int64_t)ps.popx * g.slab + ps.row * g.pitch + (sx < 0 ? 1 : g.N0 - 2)];
            else
                vals[i] = src[(int64_t)ps.pop * g.slab + ps.row * g.pitch + (sx < 0 ? g.N0 - 1 : 0)];
        }
    });
    double thm, Jd[4];  // theta - theta_ref and J in storage units
    if constexpr (std::is_same<T, float>::value) {
        // FP32 shifted storage: theta and J summed on the integer pipes
        // (f32_align in lb_device.cuh), each rounded once to FP64
        constexpr int PB = f32_align_bit<L::Q>();
        unsigned emax = 1;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) emax = max(emax, f32_exp(vals[i]));
        long long thi = 0, Ji[4] = {0, 0, 0, 0};
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const long long fv = f32_align<PB>(vals[i], emax);
            thi += fv;
            static_for<0, L::D>([&](auto Ad) {
                constexpr int a = decltype(Ad)::value;
                constexpr int ev = L::E[i][a];
                if constexpr (ev == 1) Ji[a] += fv;
                if constexpr (ev == -1) Ji[a] -= fv;
            });
        });
        const double sc = f32_scale<PB>(emax);
        thm = emax == 0xffu ? __longlong_as_double(0x7ff8000000000000ll) : i64_to_f64_rn(thi) * sc;
#pragma unroll
        for (int a = 0; a < L::D; ++a) Jd[a] = i64_to_f64_rn(Ji[a]) * sc;
    } else {
        using A = typename RecAcc<T>::type;
        A th = 0, J[4] = {0, 0, 0, 0};
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const A fv = (A)vals[i];
            th += fv;
            static_for<0, L::D>([&](auto Ad) {
                constexpr int a = decltype(Ad)::value;
                constexpr int e = L::E[i][a];
                if constexpr (e == 1) J[a] += fv;
                if constexpr (e == -1) J[a] -= fv;
            });
        });
        if constexpr (std::is_same<A, long long>::value) {  // exact integer sums, converted on the integer pipes
            thm = i64_to_f64_rn(th) * scale;
#pragma unroll
            for (int a = 0; a < L::D; ++a) Jd[a] = i64_to_f64_rn(J[a]);
        } else {
            thm = th * scale;
#pragma unroll
            for (int a = 0; a < L::D; ++a) Jd[a] = J[a];
        }
    }
    const int64_t nodes = (int64_t)g.N0 * nrow;
    const int64_t node = (row - row0) * g.N0 + x;
    const double thd = thm + r.theta_ref;
    if (theta) theta[node] = thd;
    {  // theta > 0 and finite, as bit tests on the integer pipes
        const long long tb = __double_as_longlong(thd);
        if (!(tb > 0) || ((tb >> 52) & 0x7ff) == 0x7ff) atomicOr(flag, 1);
    }
    const double cu = r.ucoef / thd;  // the storage scale is folded into ucoef and gcoef
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        const double Ja = Jd[a];
        if (grad) grad[a * nodes + node] = r.gcoef * Ja;
        if (u) u[a * nodes + node] = cu * Ja;
    }
}

template <class L, typename T, bool MIR>
static cudaError_t recover_t(lb_ctx *c, const void *src, double *th, double *gr, double *u, int *flag, int64_t row0,
                             int64_t nrow)
{
    constexpr int H = 16 / (int)sizeof(T);
    const size_t smem = (size_t)L::Q * (kTile + 2 * H) * sizeof(T);
    // up to 68 KB (D4Q33, 8-byte storage): allow more than the default 48 KB
    cudaError_t e = cudaFuncSetAttribute(recover_kernel<L, T, MIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    Recov r;
    const double scale = (c->precision == LB_FX64) ? ldexp(1.0, -c->fx_bits) : 1.0;
    // J is summed in storage units: the scale (a power of two, exact) goes into the constants
    r.ucoef = (2.0 - c->s1) * c->c * scale;
    r.gcoef = -c->s1 / (c->sigma * c->dx) * scale;
    r.theta_ref = (c->precision == LB_FP32_SHIFTED) ? c->theta_ref : 0.0;
    const int64_t blocks = nrow * ((c->geom.N0 + kTile - 1) / kTile);
    if (blocks == 0) return cudaSuccess;
    recover_kernel<L, T, MIR><<<(unsigned)blocks, kTile, smem, c->stream>>>((const T *)src, c->geom, r, scale, th,
                                                                             gr, u, flag, row0, nrow);
    return cudaGetLastError();
}

template <class L, bool MIR>
static cudaError_t recover_m(lb_ctx *c, const void *src, double *th, double *gr, double *u, int *flag, int64_t row0,
                             int64_t nrow)
{
    switch (c->precision) {
    case LB_FX64: return recover_t<L, long long, MIR>(c, src, th, gr, u, flag, row0, nrow);
    case LB_FP32_SHIFTED: return recover_t<L, float, MIR>(c, src, th, gr, u, flag, row0, nrow);
    default: return recover_t<L, double, MIR>(c, src, th, gr, u, flag, row0, nrow);
    }
}

template <class L>
static cudaError_t recover_l(lb_ctx *c, const void *src, double *th, double *gr, double *u, int *flag, int64_t row0,
                             int64_t nrow)
{
    return c->geom.mirror ? recover_m<L, true>(c, src, th, gr, u, flag, row0, nrow)
                          : recover_m<L, false>(c, src, th, gr, u, flag, row0, nrow);
}

// Self-test of the bounded wait: a barrier that nothing completes.
__global__ void staging_timeout_selftest_kernel(int *flag, unsigned long long limit_ns)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t barp = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(barp), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!mbar_wait_bounded(barp, 0, limit_ns) && threadIdx.x == 0) atomicOr(flag, 4);
}

cudaError_t launch_macros_rows(lb_ctx *c, const void *src, double *th, double *gr, double *u, int *flag, int64_t row0,
                               int64_t nrow)
{
    switch (c->d) {
    case 1: return recover_l<D1Q3>(c, src, th, gr, u, flag, row0, nrow);
    case 2: return recover_l<D2Q9>(c, src, th, gr, u, flag, row0, nrow);
    case 3: return recover_l<D3Q19>(c, src, th, gr, u, flag, row0, nrow);
    default: return recover_l<D4Q33>(c, src, th, gr, u, flag, row0, nrow);
    }
}

cudaError_t launch_macros(lb_ctx *c, const void *src, double *th, double *gr, double *u, int *flag)
{
    return launch_macros_rows(c, src, th, gr, u, flag, 0, c->geom.rows);
}

}  // namespace lbk

extern "C" lb_status lb_selftest_staging_timeout(double limit_s, void *stream, double *waited_s)
{
    if (!(limit_s > 0.0) || limit_s > 10.0) return LB_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int *dflag = nullptr;
    int flag = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&dflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        lbk::staging_timeout_selftest_kernel<<<1, 32, 0, st>>>(dflag, (unsigned long long)(limit_s * 1e9));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (waited_s) *waited_s = ms / 1e3;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(dflag);
    if (e != cudaSuccess) return LB_ECUDA;
    return (flag & 4) ? LB_ETIMEOUT : LB_OK;
}
