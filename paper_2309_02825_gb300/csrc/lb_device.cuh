// Device-side building blocks shared by the sweep, recovery, fixed-point,
// batched and adjoint kernels: compile-time loops, periodic wrap, vector
// access, the fixed-point products, the shifted pull of one
// population along x, where a pull reads from on periodic and mirror-wall
// grids (pop_source), the two gather orders, and the closed-form
// moment-space collision for D1Q3, D2Q9, D3Q19 and D4Q33
// (Eq. (distribution-f)) with the sweep kernel built from them.
#pragma once

#include "lb_internal.cuh"

namespace lbk {

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void ld_vec(const double *p, double (&a)[2])
{
    double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    a[0] = v.x;
    a[1] = v.y;
}
__device__ __forceinline__ void ld_vec(const float *p, float (&a)[4])
{
    float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    a[0] = v.x;
    a[1] = v.y;
    a[2] = v.z;
    a[3] = v.w;
}
template <typename T> __device__ __forceinline__ void ld_vec(const T *p, T (&a)[1]) { a[0] = __ldg(p); }
template <typename T> __device__ __forceinline__ void st_vec(T *p, const T (&a)[1]) { *p = a[0]; }
__device__ __forceinline__ void st_vec(float *p, const float (&a)[2])
{
    *reinterpret_cast<float2 *>(p) = make_float2(a[0], a[1]);
}
__device__ __forceinline__ void st_vec(double *p, const double (&a)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(a[0], a[1]);
}
__device__ __forceinline__ void st_vec(float *p, const float (&a)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
}
__device__ __forceinline__ void ld_vec(const float *p, float (&a)[2])
{
    float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    a[0] = v.x;
    a[1] = v.y;
}
__device__ __forceinline__ void ld_vec(const long long *p, long long (&a)[2])
{
    longlong2 v = __ldg(reinterpret_cast<const longlong2 *>(p));
    a[0] = v.x;
    a[1] = v.y;
}
__device__ __forceinline__ void st_vec(long long *p, const long long (&a)[2])
{
    *reinterpret_cast<longlong2 *>(p) = make_longlong2(a[0], a[1]);
}

// round(a * k / 2^62) for a fixed-point value a and a 62-fraction-bit constant k.
__device__ __forceinline__ long long mulfx(long long a, long long k)
{
    const __int128 p = (__int128)a * (__int128)k;
    return (long long)((p + ((__int128)1 << (kFxCoefBits - 1))) >> kFxCoefBits);
}

// The collision product: round(a k / 2^64) = floor((a k + 2^63) / 2^64) for
// a collision constant k with 64 fraction bits (a value in (-1/2, 1/2):
// |k| <= 2^63 - 2^34), from four 32 x 32-bit products in place of a 128-bit
// one.  Write a = ah 2^32 + al and k = kh 2^32 + kl with signed low words al,
// kl in [-2^31, 2^31).  Every term of a k + 2^63 but al kl is a multiple of
// 2^32, so
//   floor((a k + 2^63) / 2^32) = ah kh 2^32 + m,
//   m = ah kl + al kh + 2^31 + floor(al kl / 2^32),
// and the result is ah kh + floor(m / 2^32).  The last two terms of m,
// 2^31 + floor(al kl / 2^32), lie in [2^30, 3 2^30] and so fit one unsigned
// word; |m| <= 2^62 + 2^31 (2^31 - 4) + 3 2^30 < 2^63 (|ah| <= 2^31,
// |kh| <= 2^31 - 4).  Exact for every |a| < 2^63 - 2^31 (ah fits int32).
// Written in PTX so that each step is one instruction: the high product plus
// 2^31 is one mad.hi, and the two 64-bit accumulations are mad.wide with the
// running sum as addend (the same expression in C compiled to about 2.5x the
// instructions: separate 64-bit adds after every product).
__device__ __forceinline__ long long mulfx_c(long long a, long long k)
{
    long long r;
    asm("{\n\t"
        ".reg .b32 al, ah, kl, kh, t, c, mh, ms;\n\t"
        ".reg .b64 m, cz, mx;\n\t"
        "mov.b64 {al, ah}, %1;\n\t"
        "mov.b64 {kl, kh}, %2;\n\t"
        "shr.u32 t, kl, 31;\n\t"                    // kh += [kl < 0]: k = kh 2^32 + kl, kl signed
        "add.s32 kh, kh, t;\n\t"
        "shr.u32 t, al, 31;\n\t"                    // the same split of a
        "add.s32 ah, ah, t;\n\t"
        "mad.hi.s32 c, al, kl, -2147483648;\n\t"    // floor(al kl / 2^32) + 2^31, one unsigned word
        "cvt.u64.u32 cz, c;\n\t"
        "mad.wide.s32 m, al, kh, cz;\n\t"           // m = al kh + ah kl + c
        "mad.wide.s32 m, ah, kl, m;\n\t"
        "mov.b64 {t, mh}, m;\n\t"                   // floor(m / 2^32), sign-extended
        "shr.s32 ms, mh, 31;\n\t"
        "mov.b64 mx, {mh, ms};\n\t"
        "mad.wide.s32 %0, ah, kh, mx;\n\t"          // ah kh + floor(m / 2^32)
        "}"
        : "=l"(r)
        : "l"(a), "l"(k));
    return r;
}

// Integer -> FP64 with round-to-nearest-even, assembled from the IEEE 754
// binary64 encoding on the integer pipes (the conversion instructions issue
// at the FP64 rate, 1/64 of the integer rate on this part).  For a magnitude
// a with its leading one at bit e: the 53 bits from e down are the
// significand (implicit bit included), the bits below decide the rounding
// (above half, or exactly half with an odd significand, round up; a carry out
// of the significand moves into the exponent field by the same addition), and
// the biased exponent is e + 1023.
__device__ __forceinline__ double u64_bits_to_f64(unsigned long long a, unsigned long long sign)
{
    if (a == 0ull) return 0.0;
    const int e = 63 - __clzll((long long)a);
    unsigned long long mant, up = 0ull;
    if (e <= 52) {
        mant = a << (52 - e);
    } else {
        const int sh = e - 52;  // 1 .. 11
        mant = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        up = (rem > half || (rem == half && (mant & 1ull))) ? 1ull : 0ull;
    }
    // (e + 1022) << 52 plus the significand's implicit 2^52 gives the biased exponent e + 1023
    return __longlong_as_double((long long)((((unsigned long long)(e + 1022) << 52) + mant + up) | sign));
}

__device__ __forceinline__ double i64_to_f64_rn(long long v)
{
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    return u64_bits_to_f64(a, v < 0 ? 0x8000000000000000ull : 0ull);
}

// Exact sums of floats on the integer pipes (GB300 issues FP64 at 1/64 of its
// integer rate).  A float is m 2^(e - 150) with a 24-bit m (e its biased
// exponent, read as 1 for subnormals).  Aligned to the largest exponent E of
// the values summed, with m at bit PB, it is the integer m 2^(PB + e - E);
// f32_align_bit<N>() leaves room for N such values below 2^62, and only bits
// below 2^-(PB + 23) of the largest value are dropped (at least 2^-55; FP64
// addition rounds at 2^-53).  A sum is converted to FP64 once and scaled by
// f32_scale<PB>(E) = 2^(E - 150 - PB).
template <int N> __host__ __device__ constexpr int f32_align_bit()
{
    return 62 - 24 - (N <= 4 ? 2 : N <= 16 ? 4 : N <= 32 ? 5 : 6);
}
__device__ __forceinline__ unsigned f32_exp(float v)
{
    const unsigned e = (__float_as_uint(v) >> 23) & 0xffu;
    return e ? e : 1u;
}
template <int PB> __device__ __forceinline__ long long f32_align(float v, unsigned emax)
{
    const unsigned b = __float_as_uint(v);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | (e ? 0x800000u : 0u)) << PB;
    const unsigned sh = emax - (e ? e : 1u);
    const long long mag = (long long)(sh < 64u ? (m >> sh) : 0ull);
    return (b >> 31) ? -mag : mag;
}
template <int PB> __device__ __forceinline__ double f32_scale(unsigned emax)
{
    return __longlong_as_double((long long)(emax + 1023u - 150u - PB) << 52);  // normal for every emax <= 254
}

// Sum of N floats rounded once to FP64 (NaN if any is not finite).
template <int N> __device__ __forceinline__ double sum_f32_int(const float (&v)[N])
{
    constexpr int PB = f32_align_bit<N>();
    unsigned emax = 1;
#pragma unroll
    for (int i = 0; i < N; ++i) emax = max(emax, f32_exp(v[i]));
    long long s = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) s += f32_align<PB>(v[i], emax);
    if (emax == 0xffu) return __longlong_as_double(0x7ff8000000000000ll);
    return i64_to_f64_rn(s) * f32_scale<PB>(emax);
}

__device__ __forceinline__ double i128_to_f64_rn(__int128 v)
{
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned __int128 a = v < 0 ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(a >> 64);
    if (hi == 0ull) return u64_bits_to_f64((unsigned long long)a, sign);
    const int e = 127 - __clzll((long long)hi);  // 64 .. 127
    const int sh = e - 52;                        // 12 .. 75
    const unsigned long long mant = (unsigned long long)(a >> sh);
    const unsigned __int128 rem = a & (((unsigned __int128)1 << sh) - 1), half = (unsigned __int128)1 << (sh - 1);
    const unsigned long long up = (rem > half || (rem == half && (mant & 1ull))) ? 1ull : 0ull;
    return __longlong_as_double((long long)((((unsigned long long)(e + 1022) << 52) + mant + up) | sign));
}

// Conversion of an FP64 value to the storage type (64-bit fixed point uses
// round-to-nearest of v * 2^F).  `range` is set when a fixed-point value
// would exceed 2^61 (4x the largest theta0), leaving the sums their headroom.
template <typename T> __device__ __forceinline__ T to_store(double v, double, bool &) { return (T)v; }
template <> __device__ __forceinline__ long long to_store<long long>(double v, double fxscale, bool &range)
{
    const double s = v * fxscale;
    if (!(fabs(s) < 0x1p61)) {
        range = true;
        return 0;
    }
    return __double2ll_rn(s);
}

// Pull V consecutive values of one population along x with shift EX:
// out[k] = row[(xb + k - EX) mod N0] for the valid nodes xb + k < N0 of this
// lane (xb = x0 + V*lane).  Values for padding nodes are unspecified; loads
// past the pitch fall into the next row or the allocation's slack.
// The node x = 0 (EX = 1) reads wrow[wlo] and x = N0 - 1 (EX = -1) reads
// wrow[whi]: the same row at N0 - 1 and 0 when x is periodic, the
// x-reflected population at 1 and N0 - 2 when x has mirror walls.
// Must be called by all 32 lanes of the warp together.
template <typename T, int EX, int V = Vec<T>::V>
__device__ __forceinline__ void pull_row(const T *__restrict__ row, int x0, int lane, int N0, T (&out)[V],
                                         const T *__restrict__ wrow, int wlo, int whi)
{
    const int xb = x0 + V * lane;
    T a[V];
    ld_vec(row + xb, a);
    if constexpr (EX == 0) {
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = a[k];
    } else if constexpr (EX == 1) {
        T left = __shfl_up_sync(0xffffffffu, a[V - 1], 1);
        if (lane == 0) left = (row == wrow) ? row[xb == 0 ? wlo : xb - 1] : (xb == 0 ? wrow[wlo] : row[xb - 1]);
        out[0] = left;
#pragma unroll
        for (int k = 1; k < V; ++k) out[k] = a[k - 1];
    } else {
        T right = __shfl_down_sync(0xffffffffu, a[0], 1);
#pragma unroll
        for (int k = 0; k < V - 1; ++k) out[k] = a[k + 1];
        out[V - 1] = right;
        if (lane == 31 || xb + V >= N0) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int x = xb + k;
                if (x + 1 == N0)
                    out[k] = wrow[whi];
                else if (k == V - 1 && lane == 31 && x + 1 < N0)
                    out[k] = row[x + 1];
            }
        }
    }
}

// Row (y, z, w) of a flat row index, and the flat index of the row shifted
// by -(ey, ez, ew) with periodic wrap.  For d <= 3, w = 0 and N3 = 1.
struct RowPos {
    int y, z, w;
};
template <int D> __device__ __forceinline__ RowPos row_pos(const Geom &g, int64_t row)
{
    RowPos r;
    r.y = (int)(row % g.N1);
    if constexpr (D <= 3) {
        r.z = (int)(row / g.N1);
        r.w = 0;
    } else {
        const int64_t r2 = row / g.N1;
        r.z = (int)(r2 % g.N2);
        r.w = (int)(r2 / g.N2);
    }
    return r;
}
template <int D, int EY, int EZ, int EW>
__device__ __forceinline__ int64_t src_row(const Geom &g, const RowPos &r)
{
    const int ys = (EY == 0) ? r.y : wrapi(r.y - EY, g.N1);
    const int zs = (EZ == 0) ? r.z : wrapi(r.z - EZ, g.N2);
    if constexpr (D <= 3) {
        return (int64_t)zs * g.N1 + ys;
    } else {
        const int ws = (EW == 0) ? r.w : wrapi(r.w - EW, g.N3);
        return ((int64_t)ws * g.N2 + zs) * g.N1 + ys;
    }
}

// Source coordinate c - E on an axis of n nodes: periodic wrap, or, with
// mirror walls on nodes 0 and n - 1, reflection of -1 to 1 and of n to
// n - 2, recording the reflection in bit `bit` of m.
template <int E>
__device__ __forceinline__ int src_coord(int c, int n, bool mir, int &m, int bit)
{
    if constexpr (E == 0) {
        return c;
    } else {
        const int s = c - E;
        if (s >= 0 && s < n) return s;
        if (!mir) return s < 0 ? s + n : s - n;
        m |= bit;
        return s < 0 ? 1 : n - 2;
    }
}

// Where the pull f_i(x) = P_i(x - e_i) reads population I for target row r.
// Periodic grids: the shifted row, population I.  With mirror walls the
// doubled periodic grid (the even reflection across each wall) is folded
// back: a source row beyond a wall is the reflected row, holding the
// population whose velocity is reflected on that axis (pop).  popx is pop
// reflected on x too: the population the wall node x = 0 (or N0 - 1) pulls
// from x = 1 (or N0 - 2) when x has mirror walls.
struct PopSrc {
    int64_t row;
    int pop, popx;
};
template <class L, int I, bool MIR>
__device__ __forceinline__ PopSrc pop_source(const Geom &g, const RowPos &r)
{
    constexpr int ey = L::E[I][1], ez = L::E[I][2], ew = L::E[I][3];
    PopSrc p;
    if constexpr (!MIR) {
        p.row = src_row<L::D, ey, ez, ew>(g, r);
        p.pop = I;
        p.popx = I;
    } else {
        int m = 0;
        const int ys = src_coord<ey>(r.y, g.N1, (g.mirror >> 1) & 1u, m, 2);
        const int zs = src_coord<ez>(r.z, g.N2, (g.mirror >> 2) & 1u, m, 4);
        const int ws = src_coord<ew>(r.w, g.N3, (g.mirror >> 3) & 1u, m, 8);
        p.row = ((int64_t)ws * g.N2 + zs) * g.N1 + ys;
        p.pop = I;
        p.popx = reflect_pop<L>(I, 1);
        constexpr int nz = (ey != 0 ? 2 : 0) | (ez != 0 ? 4 : 0) | (ew != 0 ? 8 : 0);
        static_for<1, 8>([&](auto Mi) {
            constexpr int M = 2 * decltype(Mi)::value;  // subsets of the row axes y, z, w
            if constexpr ((M & ~nz) == 0) {
                if (m == M) {
                    p.pop = reflect_pop<L>(I, M);
                    p.popx = reflect_pop<L>(I, M | 1);
                }
            }
        });
    }
    return p;
}

// Gather the pre-collision f(x, n) for the V nodes of this lane, one
// population at a time (each shifted pull right after its load).  Used for
// FP64 storage, whose sweep is bound by the FP64 pipe: the lower register
// count keeps more warps resident to hide FP64 latency.
template <class L, typename T, int V = Vec<T>::V, bool MIR = false>
__device__ __forceinline__ void gather_interleaved(const T *__restrict__ src, const Geom &g, int64_t row, int x0,
                                                   int lane, T (&f)[L::Q][V])
{
    const RowPos rpos = row_pos<L::D>(g, row);
    const bool mx = MIR && (g.mirror & 1u);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::E[i][0];
        const PopSrc ps = pop_source<L, i, MIR>(g, rpos);
        const T *rp = src + (int64_t)ps.pop * g.slab + ps.row * g.pitch;
        if (!MIR || !mx) {
            pull_row<T, ex, V>(rp, x0, lane, g.N0, f[i], rp, g.N0 - 1, 0);
        } else {
            const T *rx = src + (int64_t)ps.popx * g.slab + ps.row * g.pitch;
            pull_row<T, ex, V>(rp, x0, lane, g.N0, f[i], rx, 1, g.N0 - 2);
        }
    });
}

// Gather in two phases: every 16-byte vector load of every population, and
// the one halo scalar a warp edge needs, is issued before any shuffle
// consumes a loaded value, so a warp has all q rows in flight at once.  Used
// for the HBM-bound storage types (FP32, 64-bit fixed point).
template <class L, typename T, int V = Vec<T>::V, bool MIR = false>
__device__ __forceinline__ void gather_two_phase(const T *__restrict__ src, const Geom &g, int64_t row, int x0,
                                                 int lane, T (&f)[L::Q][V])
{
    const RowPos rpos = row_pos<L::D>(g, row);
    const int xb = x0 + V * lane;
    const bool mx = MIR && (g.mirror & 1u);
    T halo[L::Q];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::E[i][0];
        const PopSrc ps = pop_source<L, i, MIR>(g, rpos);
        const T *rp = src + (int64_t)ps.pop * g.slab + ps.row * g.pitch;
        ld_vec(rp + xb, f[i]);
        halo[i] = T(0);
        if constexpr (ex == 1) {
            if constexpr (!MIR) {
                if (lane == 0) halo[i] = rp[xb == 0 ? g.N0 - 1 : xb - 1];
            } else if (lane == 0) {
                if (xb != 0)
                    halo[i] = rp[xb - 1];
                else if (!mx)
                    halo[i] = rp[g.N0 - 1];
                else
                    halo[i] = src[(int64_t)ps.popx * g.slab + ps.row * g.pitch + 1];
            }
        } else if constexpr (ex == -1) {
            const int x = xb + V - 1;
            if (lane == 31 && x + 1 < g.N0) halo[i] = rp[x + 1];
        }
    });
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::E[i][0];
        if constexpr (ex == 1) {
            T left = __shfl_up_sync(0xffffffffu, f[i][V - 1], 1);
            if (lane == 0) left = halo[i];
#pragma unroll
            for (int k = V - 1; k > 0; --k) f[i][k] = f[i][k - 1];
            f[i][0] = left;
        } else if constexpr (ex == -1) {
            T right = __shfl_down_sync(0xffffffffu, f[i][0], 1);
            if (lane == 31) right = halo[i];
#pragma unroll
            for (int k = 0; k < V - 1; ++k) f[i][k] = f[i][k + 1];
            f[i][V - 1] = right;
            if (xb + V >= g.N0) {  // the node at x = N0 - 1 pulls across the row end
                const PopSrc ps = pop_source<L, i, MIR>(g, rpos);
                const T *wp = src + (int64_t)ps.pop * g.slab + ps.row * g.pitch;
                if constexpr (MIR) {
                    if (mx) wp = src + (int64_t)ps.popx * g.slab + ps.row * g.pitch + (g.N0 - 2);
                }
#pragma unroll
                for (int k = 0; k < V; ++k)
                    if (xb + k + 1 == g.N0) f[i][k] = wp[0];
            }
        }
    });
}

// Gather for the flat lane mapping (periodic grids): one node (x, row) per
// lane, and each population read by one scalar load at its source
// (x - e_x mod N0, shifted row).  Neighbouring lanes read neighbouring
// elements, so each load is coalesced even where the warp crosses a row end;
// there are no shuffles and no per-lane halo branches.
template <class L, typename T>
__device__ __forceinline__ void gather_flat(const T *__restrict__ src, const Geom &g, int64_t row, int x,
                                            T (&f)[L::Q])
{
    const RowPos rpos = row_pos<L::D>(g, row);
    const int xl = (x == 0) ? g.N0 - 1 : x - 1;  // x - 1 and x + 1, periodic
    const int xr = (x == g.N0 - 1) ? 0 : x + 1;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::E[i][0], ey = L::E[i][1], ez = L::E[i][2], ew = L::E[i][3];
        const T *rp = src + (int64_t)i * g.slab + src_row<L::D, ey, ez, ew>(g, rpos) * g.pitch;
        f[i] = __ldg(rp + (ex == 1 ? xl : (ex == -1 ? xr : x)));
    });
}

template <class L, typename T, int V = Vec<T>::V, bool MIR = false>
__device__ __forceinline__ void gather(const T *__restrict__ src, const Geom &g, int64_t row, int x0, int lane,
                                       T (&f)[L::Q][V])
{
    // two-phase unless FP64 (FP64-pipe bound) or too many values to keep in flight
    if constexpr (std::is_same<T, double>::value || L::Q * V > 80)
        gather_interleaved<L, T, V, MIR>(src, g, row, x0, lane, f);
    else
        gather_two_phase<L, T, V, MIR>(src, g, row, x0, lane, f);
}

// The rest population is formed as theta minus all the others when the
// collision constants are rounded to float: the rounded c0, cA and wd do
// not sum to exactly one, and the resulting factor (1 + O(2^-24)) on the
// stored mass would compound step after step.  FP64 keeps the direct form
// (one FP64 instruction fewer; its constants sum to 1 within 2^-53).
template <typename T> constexpr bool kResidualRest = std::is_same<T, float>::value;

// ---------------------------------------------------------------------------
// Collision, in place on one node's q values.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void collide(D1Q3, T *f, const Coll<T> &k)
{
    const T P = f[1] + f[2];
    const T th = f[0] + P;
    const T J = f[1] - f[2];
    const T A = fma(k.k2, P, k.cA * th);
    const T B = k.k1 * J;
    if constexpr (kResidualRest<T>)
        f[0] = th - 2 * A;
    else
        f[0] = fma(-2 * k.k2, P, k.c0 * th);
    f[1] = A + B;
    f[2] = A - B;
}

template <typename T>
__device__ __forceinline__ void collide(D2Q9, T *f, const Coll<T> &k)
{
    const T a = f[1] + f[3], b = f[2] + f[4];
    const T p = f[5] + f[7], r = f[6] + f[8];
    const T Fd = p + r;
    const T th = (f[0] + a) + (b + Fd);
    const T Pxx = a + Fd, Pyy = b + Fd, Pxy = p - r;
    const T g = f[5] - f[7], h = f[8] - f[6];
    const T Jx = (f[1] - f[3]) + (g + h);
    const T Jy = (f[2] - f[4]) + (g - h);
    const T cth = k.cA * th;
    const T Ax = fma(k.k2, Pxx, cth), Bx = k.k1 * Jx;
    const T Ay = fma(k.k2, Pyy, cth), By = k.k1 * Jy;
    const T wth = k.wd * th;
    const T dp = fma(k.k3, Pxy, wth), dm = fma(-k.k3, Pxy, wth);
    if constexpr (kResidualRest<T>)
        f[0] = th - 2 * ((Ax + Ay) + (dp + dm));
    else
        f[0] = fma(-2 * k.k2, Pxx + Pyy, k.c0 * th);
    f[1] = Ax + Bx;
    f[3] = Ax - Bx;
    f[2] = Ay + By;
    f[4] = Ay - By;
    f[5] = dp;
    f[7] = dp;
    f[6] = dm;
    f[8] = dm;
}

// One coordinate plane (a, b) of D3Q19: g0..g3 are the velocities with
// (e_a, e_b) = (1,1), (-1,1), (-1,-1), (1,-1).
template <typename T> struct Plane {
    T F, P, Ja, Jb;
};
template <typename T> __device__ __forceinline__ Plane<T> plane(T g0, T g1, T g2, T g3)
{
    const T p = g0 + g2, r = g1 + g3;
    const T u = g0 - g2, v = g3 - g1;
    return {p + r, p - r, u + v, u - v};
}

template <typename T>
__device__ __forceinline__ void collide(D3Q19, T *f, const Coll<T> &k)
{
    const Plane<T> xy = plane(f[7], f[8], f[9], f[10]);
    const Plane<T> xz = plane(f[11], f[12], f[13], f[14]);
    const Plane<T> yz = plane(f[15], f[16], f[17], f[18]);
    const T ax = f[1] + f[4], ay = f[2] + f[5], az = f[3] + f[6];
    const T th = (f[0] + (ax + ay) + az) + ((xy.F + xz.F) + yz.F);
    const T Pxx = ax + (xy.F + xz.F);
    const T Pyy = ay + (xy.F + yz.F);
    const T Pzz = az + (xz.F + yz.F);
    const T Jx = (f[1] - f[4]) + (xy.Ja + xz.Ja);
    const T Jy = (f[2] - f[5]) + (xy.Jb + yz.Ja);
    const T Jz = (f[3] - f[6]) + (xz.Jb + yz.Jb);
    const T cth = k.cA * th;
    const T wth = k.wd * th;
    T rest = T(0);
    if constexpr (!kResidualRest<T>) f[0] = fma(-2 * k.k2, (Pxx + Pyy) + Pzz, k.c0 * th);
    {
        const T A = fma(k.k2, Pxx, cth), B = k.k1 * Jx;
        f[1] = A + B;
        f[4] = A - B;
        rest += A;
    }
    {
        const T A = fma(k.k2, Pyy, cth), B = k.k1 * Jy;
        f[2] = A + B;
        f[5] = A - B;
        rest += A;
    }
    {
        const T A = fma(k.k2, Pzz, cth), B = k.k1 * Jz;
        f[3] = A + B;
        f[6] = A - B;
        rest += A;
    }
    {
        const T dp = fma(k.k3, xy.P, wth), dm = fma(-k.k3, xy.P, wth);
        f[7] = dp; f[9] = dp; f[8] = dm; f[10] = dm;
        rest += dp + dm;
    }
    {
        const T dp = fma(k.k3, xz.P, wth), dm = fma(-k.k3, xz.P, wth);
        f[11] = dp; f[13] = dp; f[12] = dm; f[14] = dm;
        rest += dp + dm;
    }
    {
        const T dp = fma(k.k3, yz.P, wth), dm = fma(-k.k3, yz.P, wth);
        f[15] = dp; f[17] = dp; f[16] = dm; f[18] = dm;
        rest += dp + dm;
    }
    if constexpr (kResidualRest<T>) f[0] = th - 2 * rest;
}

// Coordinate pair p (a < b, lexicographic) of a D-dimensional lattice.
template <int D> __host__ __device__ constexpr int pair_a(int p)
{
    int a = 0, n = D - 1;
    while (p >= n) {
        p -= n;
        ++a;
        --n;
    }
    return a;
}
template <int D> __host__ __device__ constexpr int pair_b(int p)
{
    int a = 0, n = D - 1;
    while (p >= n) {
        p -= n;
        ++a;
        --n;
    }
    return a + 1 + p;
}

// The same closed-form collision for any d (used for D4Q33): the pair
// planes, axis sums and differences give theta, J_a, P_aa, P_ab.
template <class L, typename T> __device__ __forceinline__ void collide_planes(T *f, const Coll<T> &k)
{
    constexpr int D = L::D, NP = D * (D - 1) / 2, B0 = 1 + 2 * D;
    Plane<T> pl[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) pl[p] = plane(f[B0 + 4 * p], f[B0 + 4 * p + 1], f[B0 + 4 * p + 2], f[B0 + 4 * p + 3]);
    T P[D], J[D];
    T th = f[0];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        P[a] = f[1 + a] + f[1 + D + a];
        J[a] = f[1 + a] - f[1 + D + a];
        th += P[a];
    }
    static_for<0, NP>([&](auto Pi) {
        constexpr int p = decltype(Pi)::value;
        constexpr int a = pair_a<D>(p), b = pair_b<D>(p);
        th += pl[p].F;
        P[a] += pl[p].F;
        P[b] += pl[p].F;
        J[a] += pl[p].Ja;
        J[b] += pl[p].Jb;
    });
    const T cth = k.cA * th, wth = k.wd * th;
    T sumP = P[0];
#pragma unroll
    for (int a = 1; a < D; ++a) sumP += P[a];
    T rest = T(0);
    if constexpr (!kResidualRest<T>) f[0] = fma(-2 * k.k2, sumP, k.c0 * th);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T A = fma(k.k2, P[a], cth), Bq = k.k1 * J[a];
        f[1 + a] = A + Bq;
        f[1 + D + a] = A - Bq;
        rest += A;
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const T dp = fma(k.k3, pl[p].P, wth), dm = fma(-k.k3, pl[p].P, wth);
        f[B0 + 4 * p] = dp;
        f[B0 + 4 * p + 1] = dm;
        f[B0 + 4 * p + 2] = dp;
        f[B0 + 4 * p + 3] = dm;
        rest += dp + dm;
    }
    if constexpr (kResidualRest<T>) f[0] = th - 2 * rest;
}

template <typename T> __device__ __forceinline__ void collide(D4Q33, T *f, const Coll<T> &k)
{
    collide_planes<D4Q33, T>(f, k);
}

// ---------------------------------------------------------------------------
// Sweep kernel.
// ---------------------------------------------------------------------------
constexpr int kSweepThreads = 256;

// 64-bit fixed-point collisions (precision LB_FX64): exact integer moment
// sums, each product with a 64-fraction-bit relaxation constant rounded once
// (mulfx_c; the host admits only constants in (-1/2, 1/2)), and the rest
// population formed as theta minus the others, so the collision conserves
// sum f exactly.
__device__ __forceinline__ void collide(D1Q3, long long *f, const CollFx &k)
{
    const long long P = f[1] + f[2];
    const long long th = f[0] + P;
    const long long J = f[1] - f[2];
    const long long A = mulfx_c(P, k.k2) + mulfx_c(th, k.cA);
    const long long B = mulfx_c(J, k.k1);
    f[1] = A + B;
    f[2] = A - B;
    f[0] = th - 2 * A;
}

__device__ __forceinline__ void collide(D2Q9, long long *f, const CollFx &k)
{
    const long long a = f[1] + f[3], b = f[2] + f[4];
    const long long p = f[5] + f[7], r = f[6] + f[8];
    const long long Fd = p + r;
    const long long th = (f[0] + a) + (b + Fd);
    const long long Pxx = a + Fd, Pyy = b + Fd, Pxy = p - r;
    const long long g = f[5] - f[7], h = f[8] - f[6];
    const long long Jx = (f[1] - f[3]) + (g + h);
    const long long Jy = (f[2] - f[4]) + (g - h);
    const long long cth = mulfx_c(th, k.cA);
    const long long Ax = mulfx_c(Pxx, k.k2) + cth, Bx = mulfx_c(Jx, k.k1);
    const long long Ay = mulfx_c(Pyy, k.k2) + cth, By = mulfx_c(Jy, k.k1);
    const long long wth = mulfx_c(th, k.wd);
    const long long B3 = mulfx_c(Pxy, k.k3);
    const long long dp = wth + B3, dm = wth - B3;
    f[1] = Ax + Bx;
    f[3] = Ax - Bx;
    f[2] = Ay + By;
    f[4] = Ay - By;
    f[5] = dp;
    f[7] = dp;
    f[6] = dm;
    f[8] = dm;
    f[0] = th - 2 * ((Ax + Ay) + (dp + dm));
}

__device__ __forceinline__ void collide(D3Q19, long long *f, const CollFx &k)
{
    const Plane<long long> xy = plane(f[7], f[8], f[9], f[10]);
    const Plane<long long> xz = plane(f[11], f[12], f[13], f[14]);
    const Plane<long long> yz = plane(f[15], f[16], f[17], f[18]);
    const long long ax = f[1] + f[4], ay = f[2] + f[5], az = f[3] + f[6];
    const long long th = (f[0] + (ax + ay) + az) + ((xy.F + xz.F) + yz.F);
    const long long Pxx = ax + (xy.F + xz.F);
    const long long Pyy = ay + (xy.F + yz.F);
    const long long Pzz = az + (xz.F + yz.F);
    const long long Jx = (f[1] - f[4]) + (xy.Ja + xz.Ja);
    const long long Jy = (f[2] - f[5]) + (xy.Jb + yz.Ja);
    const long long Jz = (f[3] - f[6]) + (xz.Jb + yz.Jb);
    const long long cth = mulfx_c(th, k.cA);
    const long long wth = mulfx_c(th, k.wd);
    long long axis = 0, diag = 0;
    {
        const long long A = mulfx_c(Pxx, k.k2) + cth, B = mulfx_c(Jx, k.k1);
        f[1] = A + B;
        f[4] = A - B;
        axis += A;
    }
    {
        const long long A = mulfx_c(Pyy, k.k2) + cth, B = mulfx_c(Jy, k.k1);
        f[2] = A + B;
        f[5] = A - B;
        axis += A;
    }
    {
        const long long A = mulfx_c(Pzz, k.k2) + cth, B = mulfx_c(Jz, k.k1);
        f[3] = A + B;
        f[6] = A - B;
        axis += A;
    }
    {
        const long long B = mulfx_c(xy.P, k.k3), dp = wth + B, dm = wth - B;
        f[7] = dp; f[9] = dp; f[8] = dm; f[10] = dm;
        diag += dp + dm;
    }
    {
        const long long B = mulfx_c(xz.P, k.k3), dp = wth + B, dm = wth - B;
        f[11] = dp; f[13] = dp; f[12] = dm; f[14] = dm;
        diag += dp + dm;
    }
    {
        const long long B = mulfx_c(yz.P, k.k3), dp = wth + B, dm = wth - B;
        f[15] = dp; f[17] = dp; f[16] = dm; f[18] = dm;
        diag += dp + dm;
    }
    f[0] = th - 2 * (axis + diag);
}

// Any d (used for D4Q33): pair planes, exact integer moment sums, rounded
// products, rest population = theta minus the others.
__device__ __forceinline__ void collide(D4Q33, long long *f, const CollFx &k)
{
    constexpr int D = 4, NP = 6, B0 = 1 + 2 * D;
    Plane<long long> pl[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) pl[p] = plane(f[B0 + 4 * p], f[B0 + 4 * p + 1], f[B0 + 4 * p + 2], f[B0 + 4 * p + 3]);
    long long P[D], J[D];
    long long th = f[0];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        P[a] = f[1 + a] + f[1 + D + a];
        J[a] = f[1 + a] - f[1 + D + a];
        th += P[a];
    }
    static_for<0, NP>([&](auto Pi) {
        constexpr int p = decltype(Pi)::value;
        constexpr int a = pair_a<D>(p), b = pair_b<D>(p);
        th += pl[p].F;
        P[a] += pl[p].F;
        P[b] += pl[p].F;
        J[a] += pl[p].Ja;
        J[b] += pl[p].Jb;
    });
    const long long cth = mulfx_c(th, k.cA), wth = mulfx_c(th, k.wd);
    long long rest = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const long long A = mulfx_c(P[a], k.k2) + cth, Bq = mulfx_c(J[a], k.k1);
        f[1 + a] = A + Bq;
        f[1 + D + a] = A - Bq;
        rest += A;
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const long long Bq = mulfx_c(pl[p].P, k.k3), dp = wth + Bq, dm = wth - Bq;
        f[B0 + 4 * p] = dp;
        f[B0 + 4 * p + 1] = dm;
        f[B0 + 4 * p + 2] = dp;
        f[B0 + 4 * p + 3] = dm;
        rest += dp + dm;
    }
    f[0] = th - 2 * rest;
}


// Threads per block of the sweep: 128 for the HBM-bound storage types
// (more, smaller blocks balance the SMs better), 256 for FP64.
template <typename T> __host__ __device__ constexpr int sweep_threads() { return std::is_same<T, double>::value ? 256 : 128; }

// K is the collision-constant type; the matching collide() overload (float,
// double or 64-bit fixed point) is picked by overload resolution.
// MIR: the grid has mirror walls on some axis (g.mirror); the periodic
// instantiation carries none of that logic.
template <class L, typename T, class K, bool MIR = false>
__global__ void __launch_bounds__(sweep_threads<T>()) sweep_kernel(const T *__restrict__ src,
                                                                   T *__restrict__ dst, Geom g, K k)
{
    constexpr int V = lane_width<L, T>();
    constexpr int TH = sweep_threads<T>();
    const int lane = threadIdx.x & 31;
    const int64_t seg = (int64_t)blockIdx.x * (TH / 32) + (threadIdx.x >> 5);
    if (seg >= g.nseg) return;  // warp-uniform
    const int64_t row = seg / g.seg_per_row;
    const int x0 = (int)(seg - row * g.seg_per_row) * (32 * V);

    T f[L::Q][V];
    gather<L, T, V, MIR>(src, g, row, x0, lane, f);

#pragma unroll
    for (int v = 0; v < V; ++v) {
        T n[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) n[i] = f[i][v];
        collide(L{}, n, k);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) f[i][v] = n[i];
    }
    if constexpr (std::is_same<K, CollFxR>::value) {
        // |v| < 2^61 iff v + 2^61 lies in [0, 2^62): only the high word of
        // the sum changes, so OR the high words + 2^29 and test bits 30, 31
        unsigned acc = 0u;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (x0 + V * lane + v < g.N0) {
#pragma unroll
                for (int i = 0; i < L::Q; ++i) acc |= (unsigned)((unsigned long long)f[i][v] >> 32) + 0x20000000u;
            }
        }
        if (__any_sync(0xffffffffu, acc >= 0x40000000u) && lane == 0) atomicOr(k.range, 1);
    }

    if (x0 + V * lane >= g.pitch) return;  // beyond the row: loads only
    T *dp = dst + row * g.pitch + x0 + V * lane;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) st_vec(dp + (int64_t)i * g.slab, f[i]);
}

// Node `q` of the flat mapping (row-major over the N0 nodes of each row):
// its row and x.  Lanes past the last node take the last one (loads only;
// they never store).
__device__ __forceinline__ void flat_node(const Geom &g, int64_t q, int64_t &row, int &x)
{
    const unsigned n = (unsigned)(g.rows * g.N0);  // < 2^31 wherever the flat mapping is used
    const unsigned qc = q < (int64_t)n ? (unsigned)q : n - 1u;
    const unsigned r = qc / (unsigned)g.N0;
    row = r;
    x = (int)(qc - r * (unsigned)g.N0);
}

// The sweep with the flat mapping, for periodic 4D grids with 8-byte states
// whose rows do not fill whole warps (Example 4's 20 .. 50 nodes per row):
// same pull and collision per node as sweep_kernel.  Every lane works (the
// row-segment mapping leaves up to 38 % of them idle at N0 = 20 .. 50), and
// with one node per lane and no halo the kernel holds 80-90 registers instead
// of 128-164, so more warps stay resident.
template <class L, typename T, class K>
__global__ void __launch_bounds__(sweep_threads<T>()) sweep_flat_kernel(const T *__restrict__ src,
                                                                        T *__restrict__ dst, Geom g, K k)
{
    constexpr int TH = sweep_threads<T>();
    const int lane = threadIdx.x & 31;
    const int64_t seg = (int64_t)blockIdx.x * (TH / 32) + (threadIdx.x >> 5);
    if (seg >= g.fseg) return;  // warp-uniform
    const int64_t q = seg * 32 + lane;
    int64_t row;
    int x;
    flat_node(g, q, row, x);
    T f[L::Q];
    gather_flat<L, T>(src, g, row, x, f);
    collide(L{}, f, k);
    if constexpr (std::is_same<K, CollFxR>::value) {
        unsigned acc = 0u;  // |v| < 2^61 check, as in sweep_kernel
        if (q < g.rows * g.N0) {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) acc |= (unsigned)((unsigned long long)f[i] >> 32) + 0x20000000u;
        }
        if (__any_sync(0xffffffffu, acc >= 0x40000000u) && lane == 0) atomicOr(k.range, 1);
    }
    if (q >= g.rows * g.N0) return;  // past the last node: loads only
    T *dp = dst + row * g.pitch + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) dp[(int64_t)i * g.slab] = f[i];
}

}  // namespace lbk
