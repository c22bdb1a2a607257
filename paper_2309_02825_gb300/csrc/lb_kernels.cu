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
// Initialisation (first two terms of Eq. (f-feq-o5), closed form):
//   f_0 = w0 th,  f(+-e_a) = w1 th -+ iax d_a th,  f(diag e) = wd th - idg (e . grad th),
// stored in P form, P_0(y, i) = f_i(y + e_i, 0).  One thread per node x
// forms all q values of x once and stores f_i(x) at y = x - e_i (periodic
// wrap).  On an axis with mirror walls a destination beyond a wall is not
// stored (the doubled grid's ghost), and a thread next to a wall (x_a = 1
// with e_ia = +1, or x_a = N_a - 2 with e_ia = -1) also stores f_i(x) in
// the wall node's slot of the reflected population: that slot's source lies
// beyond the wall, at the mirror image of x.  Every stored slot has exactly
// one writer.  The wall-normal gradient component is odd across the wall, so
// on a wall node it is taken as zero.
//
// FXI (64-bit fixed point formed in integers): theta and dx * grad theta are
// converted to fixed point once per node, every product with a constant is
// a rounded 64x62-bit product, and the rest population is theta minus the
// others, so sum_i f_i(x) = round(theta0(x) 2^F) exactly.
// ---------------------------------------------------------------------------
// round(v 2^F) to nearest, ties to even, from the fields of the IEEE double
// v in integer arithmetic (v 2^F is exact; only its rounding to an integer is
// done here).  Sets `range` when |v 2^F| >= 2^61, NaN and infinities included.
__device__ __forceinline__ long long fx_round(double v, int F, bool &range)
{
    const long long bits = __double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ff);
    const long long mant = (bits & ((1ll << 52) - 1)) | (e ? (1ll << 52) : 0ll);
    const int sh = (e ? e : 1) - 1075 + F;  // |v| 2^F = mant 2^sh
    if (e == 0x7ff || sh > 8) {             // mant >= 2^52: sh >= 9 means >= 2^61
        range = true;
        return 0;
    }
    long long r;
    if (sh >= 0) {
        r = mant << sh;
    } else if (sh < -53) {
        r = 0;  // below one half
    } else {
        const int k = -sh;
        const long long q = mant >> k, rem = mant & ((1ll << k) - 1), half = 1ll << (k - 1);
        r = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
    }
    return bits < 0 ? -r : r;
}

template <class L, typename T, bool FXI>
__global__ void init_kernel(T *__restrict__ dst, Geom g, InitK K, const double *__restrict__ theta0,
                            const double *__restrict__ grad, int *__restrict__ flag)
{
    constexpr int D = L::D, Q = L::Q;
    const int64_t nodes = (int64_t)g.N0 * g.rows;
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nodes) return;
    // coordinates in 32-bit arithmetic (nodes <= 2^31)
    const unsigned nd = (unsigned)node;
    int c[4];
    const unsigned rw = nd / (unsigned)g.N0;
    c[0] = (int)(nd - rw * (unsigned)g.N0);
    const unsigned r2 = rw / (unsigned)g.N1;
    c[1] = (int)(rw - r2 * (unsigned)g.N1);
    const unsigned r3 = r2 / (unsigned)g.N2;
    c[2] = (int)(r2 - r3 * (unsigned)g.N2);
    c[3] = (int)r3;
    const int n[4] = {g.N0, g.N1, g.N2, g.N3};

    // checks on the bit patterns (integer pipes): theta > 0 and finite, a
    // finite gradient (exponent field not all ones)
    const double th = theta0[node];
    const long long tb = __double_as_longlong(th);
    double gr[D];
    bool bad = !(tb > 0) || ((tb >> 52) & 0x7ff) == 0x7ff;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        gr[a] = grad[a * nodes + node];
        bad |= ((__double_as_longlong(gr[a]) >> 52) & 0x7ff) == 0x7ff;
        if (((g.mirror >> a) & 1u) && (c[a] == 0 || c[a] == n[a] - 1)) gr[a] = 0.0;
    }
    if (bad) atomicOr(flag, 1);

    T val[Q];
    bool range = false;
    if constexpr (FXI) {
        const long long t = fx_round(th, K.fx_bits, range);
        long long G[D];
#pragma unroll
        for (int a = 0; a < D; ++a) G[a] = fx_round(gr[a] * K.gscale, 0, range);
        const long long W1 = mulfx(t, K.w1k), WD = mulfx(t, K.wdk);
        long long rest = 0;
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int nz = (L::E[i][0] != 0) + (L::E[i][1] != 0) + (L::E[i][2] != 0) + (L::E[i][3] != 0);
            long long v;
            if constexpr (nz == 1) {
                constexpr int a = (L::E[i][0] != 0) ? 0 : ((L::E[i][1] != 0) ? 1 : ((L::E[i][2] != 0) ? 2 : 3));
                constexpr int ea = L::E[i][a];
                const long long A = mulfx(G[a], K.iak);
                v = (ea > 0) ? W1 - A : W1 + A;
            } else {
                constexpr int a = (L::E[i][0] != 0) ? 0 : ((L::E[i][1] != 0) ? 1 : 2);
                constexpr int b = (L::E[i][3] != 0) ? 3 : ((L::E[i][2] != 0 && a < 2) ? 2 : 1);
                constexpr int ea = L::E[i][a], eb = L::E[i][b];
                // e . (dx grad) = +-(G_a + G_b) or +-(G_a - G_b); one rounded product per pair and sign
                const long long P = mulfx(ea == eb ? G[a] + G[b] : G[a] - G[b], K.wdk);
                v = (ea > 0) ? WD - P : WD + P;
            }
            if (!(v < (1ll << 61) && v > -(1ll << 61))) range = true;
            val[i] = v;
            rest += v;
        });
        val[0] = t - rest;
    } else if constexpr (std::is_same<T, float>::value) {
        // FP32 shifted storage: f_i - w_i theta_ref formed from theta0 - theta_ref
        // and the gradient terms, each shared term computed once (the float
        // rounding of the stored value dominates; FP64 issues at 1/64 of the
        // FP32 rate on this part, so the FP64 operations per node are kept few)
        const double dth = th - K.theta_ref;
        const double b0 = K.w0 * dth, b1 = K.w1 * dth, bd = K.wd * dth;
        double ga[D];
#pragma unroll
        for (int a = 0; a < D; ++a) ga[a] = K.iax * gr[a];
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ex = L::E[i][0], ey = L::E[i][1], ez = L::E[i][2], ew = L::E[i][3];
            constexpr int nz = (ex != 0) + (ey != 0) + (ez != 0) + (ew != 0);
            double v;
            if constexpr (nz == 0) {
                v = b0;
            } else if constexpr (nz == 1) {
                constexpr int a = (ex != 0) ? 0 : ((ey != 0) ? 1 : ((ez != 0) ? 2 : 3));
                constexpr int sgn = (ex != 0) ? ex : ((ey != 0) ? ey : ((ez != 0) ? ez : ew));
                v = sgn > 0 ? b1 - ga[a] : b1 + ga[a];
            } else {
                double edg = 0.0;
                if constexpr (ex != 0) edg += (double)ex * gr[0];
                if constexpr (ey != 0) edg += (double)ey * gr[1];
                if constexpr (ez != 0) edg += (double)ez * gr[2];
                if constexpr (ew != 0) edg += (double)ew * gr[3];
                v = fma(-K.idg, edg, bd);
            }
            val[i] = (T)v;
        });
    } else {
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ex = L::E[i][0], ey = L::E[i][1], ez = L::E[i][2], ew = L::E[i][3];
            constexpr int nz = (ex != 0) + (ey != 0) + (ez != 0) + (ew != 0);
            double v;
            if constexpr (nz == 0) {
                v = K.w0 * th;
                v -= K.w0 * K.theta_ref;
            } else if constexpr (nz == 1) {
                constexpr int a = (ex != 0) ? 0 : ((ey != 0) ? 1 : ((ez != 0) ? 2 : 3));
                constexpr int sgn = (ex != 0) ? ex : ((ey != 0) ? ey : ((ez != 0) ? ez : ew));
                v = K.w1 * th - (double)sgn * K.iax * gr[a];
                v -= K.w1 * K.theta_ref;
            } else {
                double edg = 0.0;
                if constexpr (ex != 0) edg += (double)ex * gr[0];
                if constexpr (ey != 0) edg += (double)ey * gr[1];
                if constexpr (ez != 0) edg += (double)ez * gr[2];
                if constexpr (ew != 0) edg += (double)ew * gr[3];
                v = K.wd * th - K.idg * edg;
                v -= K.wd * K.theta_ref;
            }
            val[i] = to_store<T>(v, K.fxscale, range);
        });
    }
    if (range) atomicOr(flag, 2);

    if (!g.mirror) {
        // periodic: destination offset = sum over axes of one of three wrapped
        // offsets (shift -1, 0, +1), formed once per node
        int64_t off[4][3];
        int64_t stride = 1;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int dn = c[a] == 0 ? n[a] - 1 : c[a] - 1;  // x_a - 1
            const int up = c[a] == n[a] - 1 ? 0 : c[a] + 1;  // x_a + 1
            off[a][0] = (int64_t)up * stride;                // e = -1 stores at x_a + 1
            off[a][1] = (int64_t)c[a] * stride;
            off[a][2] = (int64_t)dn * stride;                // e = +1 stores at x_a - 1
            stride *= (a == 0) ? (int64_t)g.pitch : (int64_t)n[a];
        }
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const int64_t at = off[0][L::E[i][0] + 1] + off[1][L::E[i][1] + 1] + off[2][L::E[i][2] + 1] +
                               off[3][L::E[i][3] + 1];
            dst[(int64_t)i * g.slab + at] = val[i];
        });
        return;
    }
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int E0 = L::E[i][0], E1 = L::E[i][1], E2 = L::E[i][2], E3 = L::E[i][3];
        const int ev[4] = {E0, E1, E2, E3};
        int y[4];
        bool ghost = false;
        unsigned near = 0;  // axes where x is next to a wall it streams onto
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int e = ev[a];
            int v = c[a] - e;
            if (e != 0 && ((g.mirror >> a) & 1u)) {
                if (v < 0 || v >= n[a]) ghost = true;
                if ((e > 0 && c[a] == 1) || (e < 0 && c[a] == n[a] - 2)) near |= 1u << a;
            } else if (v < 0) {
                v += n[a];
            } else if (v >= n[a]) {
                v -= n[a];
            }
            y[a] = v;
        }
        if (ghost) return;
        const int64_t at = (((int64_t)y[3] * g.N2 + y[2]) * g.N1 + y[1]) * g.pitch + y[0];
        dst[(int64_t)i * g.slab + at] = val[i];
        if (near) {
            constexpr int nzm = (E0 != 0 ? 1 : 0) | (E1 != 0 ? 2 : 0) | (E2 != 0 ? 4 : 0) | (E3 != 0 ? 8 : 0);
            static_for<1, 16>([&](auto Mi) {
                constexpr int M = decltype(Mi)::value;
                if constexpr ((M & ~nzm) == 0) {
                    if ((M & ~near) == 0) dst[(int64_t)reflect_pop<L>(i, M) * g.slab + at] = val[i];
                }
            });
        }
    });
}

// Fourth-order central difference of theta along each axis: periodic, or,
// on an axis with mirror walls (bit a of mirror), the even reflection of
// theta across the wall nodes (theta(-k) = theta(k)).
__global__ void fd4_kernel(const double *__restrict__ th, double *__restrict__ grad, int d, int N0, int N1,
                           int N2, int N3, unsigned mirror, double inv12dx)
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
            const int t = c[a] + off[k];
            if ((mirror >> a) & 1u)
                c[a] = t < 0 ? -t : (t >= n[a] ? 2 * (n[a] - 1) - t : t);
            else
                c[a] = (t % n[a] + n[a]) % n[a];
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

// Weight of a row of nodes in the conserved total: 1/2 per mirror wall of
// the y, z, w axes the row lies on (the doubled periodic grid holds interior
// nodes twice, wall nodes once); the x walls halve the row's first and last
// node.
__device__ __forceinline__ double row_wall_weight(const Geom &g, int64_t row)
{
    double wt = 1.0;
    const int y = (int)(row % g.N1);
    const int64_t r2 = row / g.N1;
    const int z = (int)(r2 % g.N2);
    const int w = (int)(r2 / g.N2);
    if ((g.mirror & 2u) && (y == 0 || y == g.N1 - 1)) wt *= 0.5;
    if ((g.mirror & 4u) && (z == 0 || z == g.N2 - 1)) wt *= 0.5;
    if ((g.mirror & 8u) && (w == 0 || w == g.N3 - 1)) wt *= 0.5;
    return wt;
}

template <typename T> struct SumAcc {
    using type = double;
};
template <> struct SumAcc<long long> {
    using type = __int128;  // exact: fixed-point values add without rounding
};
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(__int128 v)
{
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return (double)hi * 0x1p64 + (double)lo;
}

// Sum of the stored state over populations and valid nodes (weighted by
// the wall weights when the grid has mirror walls): one warp per row of
// one population, aligned 16-byte vector loads along the row.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) sum_state_kernel(const T *__restrict__ src, Geom g, int q,
                                                                double scale, double *__restrict__ partial)
{
    constexpr int V = Vec<T>::V;
    typename SumAcc<T>::type acc = 0;
    double accw = 0.0;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // rows of the sum: g.rows per population (a sub-range of the grid's rows
    // when src starts past row 0), populations g.slab values apart
    const int64_t nrows = (int64_t)q * g.rows;
    constexpr int U = 4;  // vectors in flight per lane
    for (int64_t r = warp; r < nrows; r += nwarps) {
        const int64_t pop = r / g.rows, row = r - pop * g.rows;
        const T *rowp = src + pop * g.slab + row * g.pitch;
        const double rw = g.mirror ? row_wall_weight(g, row) : 1.0;
        for (int x0 = lane * V; x0 < g.N0; x0 += U * 32 * V) {
            T a[U][V];
#pragma unroll
            for (int j = 0; j < U; ++j)
                if (x0 + j * 32 * V < g.N0) ld_vec(rowp + x0 + j * 32 * V, a[j]);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if constexpr (std::is_same<T, float>::value) {
                    // a whole vector of floats: one integer-pipe sum and one FP64 addition
                    if (!g.mirror && x0 + j * 32 * V + V <= g.N0) {
                        acc += sum_f32_int(a[j]);
                        continue;
                    }
                }
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const int x = x0 + j * 32 * V + k;
                    if (x >= g.N0) continue;
                    if (!g.mirror) {
                        acc += a[j][k];
                    } else {
                        const double xw = ((g.mirror & 1u) && (x == 0 || x == g.N0 - 1)) ? 0.5 : 1.0;
                        accw += (double)a[j][k] * (rw * xw);
                    }
                }
            }
        }
    }
    Acc<1> a{{(to_double(acc) + accw) * scale}};
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
    // max |err| on the integer pipes: for non-negative doubles the bit
    // patterns order like the values (a NaN error shows in the RMSE sums)
    long long mx[D + 1];
#pragma unroll
    for (int c = 0; c <= D; ++c) mx[c] = 0;
    constexpr long long kAbs = 0x7fffffffffffffffll;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nodes;
         n += (int64_t)gridDim.x * blockDim.x) {
        const double t = th[n], te = eth[n];
        const double e = t - te;
        a.v[0] = fma(e, e, a.v[0]);
        mx[0] = max(mx[0], __double_as_longlong(e) & kAbs);
        a.v[2] = fma(te, te, a.v[2]);
        a.v[NS - 1] += t;
        if (u) {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double uv = u[c * nodes + n], ue = eu[c * nodes + n];
                const double eu2 = uv - ue;
                a.v[3 * (c + 1) + 0] = fma(eu2, eu2, a.v[3 * (c + 1) + 0]);
                mx[c + 1] = max(mx[c + 1], __double_as_longlong(eu2) & kAbs);
                a.v[3 * (c + 1) + 2] = fma(ue, ue, a.v[3 * (c + 1) + 2]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c <= D; ++c) a.v[3 * c + 1] = __longlong_as_double(mx[c]);
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
    const bool flat = sweep_flat(c->geom, L::D, (int)sizeof(T));
    const unsigned nb = (unsigned)(((flat ? c->geom.fseg : c->geom.nseg) + TH / 32 - 1) / (TH / 32));
    if constexpr (L::D == 4 && sizeof(T) == 8) {
        if (flat) {
            sweep_flat_kernel<L, T, Coll<T>><<<nb, TH, 0, c->stream>>>((const T *)src, (T *)dst, c->geom,
                                                                       make_coll<T>(*c));
            return cudaGetLastError();
        }
    }
    if (c->geom.mirror)
        sweep_kernel<L, T, Coll<T>, true><<<nb, TH, 0, c->stream>>>(
            (const T *)src, (T *)dst, c->geom, make_coll<T>(*c));
    else
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
        theta0, grad, c->d, (int)c->N[0], (int)c->N[1], (int)c->N[2], (int)c->N[3], c->geom.mirror,
        1.0 / (12.0 * c->dx));
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
    K.gscale = c->dx * K.fxscale;
    K.fx_bits = c->fx_bits;
    const unsigned nb = (unsigned)((c->nodes + 255) / 256);
    if constexpr (std::is_same<T, long long>::value) {
        // integer formation needs every constant inside the 62-bit range and
        // a total weight that keeps the rest population's sum below 2^61
        const double ia = K.iax / c->dx;
        const double wmass = fabs(c->w0) + 2.0 * d * fabs(c->w1) + 2.0 * d * (d - 1.0) * fabs(wd);
        if (fabs(ia) < 1.5 && fabs(c->w1) < 1.0 && fabs(wd) < 1.0 && wmass <= 4.0) {
            K.w1k = llrint(ldexp(c->w1, kFxCoefBits));
            K.wdk = llrint(ldexp(wd, kFxCoefBits));
            K.iak = llrint(ldexp(ia, kFxCoefBits));
            init_kernel<L, T, true><<<nb, 256, 0, c->stream>>>((T *)c->f[c->cur], c->geom, K, theta0, grad, flag);
            return cudaGetLastError();
        }
    }
    K.w1k = K.wdk = K.iak = 0;
    init_kernel<L, T, false><<<nb, 256, 0, c->stream>>>((T *)c->f[c->cur], c->geom, K, theta0, grad, flag);
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

cudaError_t launch_sum_state_rows(lb_ctx *c, const void *src, double *out_dev, int64_t row0, int64_t nrow)
{
    const int nb = c->scratch_blocks;
    Geom g = c->geom;  // rows row0 .. row0 + nrow - 1 of every population (no walls on a sub-range)
    g.rows = nrow;
    if (row0 != 0 || nrow != c->geom.rows) g.mirror = 0;
    const int64_t off = row0 * g.pitch;
    if (c->precision == LB_FP64)
        sum_state_kernel<double><<<nb, kRedThreads, 0, c->stream>>>((const double *)src + off, g, c->q, 1.0,
                                                                     c->scratch);
    else if (c->precision == LB_FX64)
        sum_state_kernel<long long><<<nb, kRedThreads, 0, c->stream>>>(
            (const long long *)src + off, g, c->q, ldexp(1.0, -c->fx_bits), c->scratch);
    else
        sum_state_kernel<float><<<nb, kRedThreads, 0, c->stream>>>((const float *)src + off, g, c->q, 1.0,
                                                                    c->scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_kernel<<<1, kRedThreads, 0, c->stream>>>(c->scratch, nb, 1, 0u, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_sum_state(lb_ctx *c, const void *src, double *out_dev)
{
    return launch_sum_state_rows(c, src, out_dev, 0, c->geom.rows);
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
