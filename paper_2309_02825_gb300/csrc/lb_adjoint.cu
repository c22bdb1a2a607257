// Discrete adjoint of the MRT-LB forward map (include/lb_adjoint.h).
//
// Notation: f_n(x) is the pre-collision distribution at step n, stored in
// P form (P_{n+1}(x) = K f_n(x), f_n(x)_i = P_n(x - e_i)_i); phi_n(x) =
// dL/df_n(x) is held aligned at x in FP64.  Then
//   phi_n(x) = K^T lambda_{n+1}(x),  lambda_{n+1}(x)_i = phi_{n+1}(x + e_i)_i,
//   dL/deps += lambda_{n+1}(x) . (dK/deps) f_n(x).
// K^T is written in moment form by transposing the closed-form collision:
// with Lt = c0 l0 + cA sum_axis l + wd sum_diag l, Laa = k2 (l_{+a} + l_{-a}
// - 2 l0), Ja = k1 (l_{+a} - l_{-a}), Lab = k3 sum_{diag(a,b)} sa sb l,
//   (K^T l)_j = Lt + sum_a e_ja^2 Laa + sum_a e_ja Ja + sum_{a<b} e_ja e_jb Lab.
// The collision is linear in its constants, so lambda . (dK/deps) f is the
// same bilinear form with the eps-derivatives of the constants: the lambda
// channels of K^T (l0, l_{+a} +- l_{-a}, the plane sums) against the
// moments of f (theta, J_a, P_aa, P_ab), a handful of products per node.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/lb_adjoint.h"
#include "lb_device.cuh"

namespace lbk {

constexpr int kAdjQ = 19;

struct AdjK {
    Coll<double> k;   // collision constants
    Coll<double> kd;  // their eps-derivatives
    Coll<float> kf, kdf;  // the same in float, for the FP32 reverse pass of FP32-shifted states
    double scale;     // stored value -> f: f_i = v * scale + shift[i]
    double shift[kAdjQ];
    double mshift_th, mshift_paa;  // the shift's moments: theta_ref and sigma theta_ref
    float mshift_th_f, mshift_paa_f;
    // Fixed-point reverse pass (64-bit fixed-point states): the adjoint fields
    // hold round(phi 2^G); aunit = 2^-G.  K^T uses the collision constants with
    // kFxCoefBits fraction bits (c0k .. wdk); the eps-term uses the FP64
    // eps-derivatives scaled by 2^-(F+G) (kdx), F the state's fraction bits.
    long long c0k, cAk, wdk, k1k, k2k, k3k;
    double aunit;
    Coll<double> kdx;
    double ucoef, ducoef;                      // (2 - s1) c and d/deps
    double w[kAdjQ], dw[kAdjQ];                // weights and d/deps
    double iax, idg, diax, didg;               // initialisation operator and d/deps
    double inv12dx;
};

template <typename T> __device__ __forceinline__ double to_f(T v, double scale) { return (double)v * scale; }

// Reverse pull: out[k] = phi(x + e_i) for the V nodes of this lane.
template <class L, typename A>
__device__ __forceinline__ void gather_rev(const A *__restrict__ src, const Geom &g, int64_t row, int x0, int lane,
                                           A (&f)[L::Q][2])
{
    const int y = (int)(row % g.N1);
    const int z = (int)(row / g.N1);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::E[i][0], ey = L::E[i][1], ez = L::E[i][2];
        const int ys = (ey == 0) ? y : wrapi(y + ey, g.N1);
        const int zs = (ez == 0) ? z : wrapi(z + ez, g.N2);
        const A *rp = src + (int64_t)i * g.slab + ((int64_t)zs * g.N1 + ys) * g.pitch;
        pull_row<A, -ex, 2>(rp, x0, lane, g.N0, f[i], rp, g.N0 - 1, 0);
    });
}

// Reverse pull on a grid with mirror walls.  The forward pull reads the
// stored slot P_j(y) from the node x = y + e_j: f_j(x) reads it, and so does
// f_{R_B(j)}(x) for every set B of walls that e_j points into at x (x on the
// wall node of axis a in B, e_ja pointing out of the domain), because a pull
// across a wall reads the reflected population.  The transpose therefore
// gathers lambda_j(y) = sum over those B of phi_{R_B(j)}(x), and zero when x
// lies beyond a wall (such slots are never read).  Plain loads, one node at a
// time: only grids with walls take this path.
__device__ __forceinline__ int adj_src(int c, int e, int n, bool mir, bool &ghost, int &wall, int bit)
{
    if (e == 0) return c;
    const int s = c + e;
    if (s >= 0 && s < n) {
        if (mir && ((e < 0 && s == 0) || (e > 0 && s == n - 1))) wall |= bit;
        return s;
    }
    if (!mir) return s < 0 ? s + n : s - n;
    ghost = true;
    return 0;
}

template <class L, typename A>
__device__ __forceinline__ void gather_rev_walls(const A *__restrict__ src, const Geom &g, int64_t row, int x0,
                                                 int lane, A (&f)[L::Q][2])
{
    const int y = (int)(row % g.N1);
    const int z = (int)(row / g.N1);
    const int xb = x0 + 2 * lane;
    static_for<0, L::Q>([&](auto I) {
        constexpr int j = decltype(I)::value;
        constexpr int ex = L::E[j][0], ey = L::E[j][1], ez = L::E[j][2];
        constexpr int nz = (ey != 0 ? 2 : 0) | (ez != 0 ? 4 : 0);  // row axes e_j moves along
        bool ghost = false;
        int wall = 0;  // bit a: the wall of axis a at the source node
        const int ys = adj_src(y, ey, g.N1, (g.mirror >> 1) & 1u, ghost, wall, 2);
        const int zs = adj_src(z, ez, g.N2, (g.mirror >> 2) & 1u, ghost, wall, 4);
        const int64_t rbase = ((int64_t)zs * g.N1 + ys) * g.pitch;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            A acc = 0;
            if (!ghost && xb + v < g.N0) {
                bool gx = false;
                int wx = 0;
                const int xs = adj_src(xb + v, ex, g.N0, g.mirror & 1u, gx, wx, 1);
                if (!gx) {
                    static_for<0, 8>([&](auto Mi) {
                        constexpr int M = 2 * decltype(Mi)::value;  // subsets of the row axes
                        if constexpr ((M & ~nz) == 0) {
                            if ((M & ~wall) == 0) {
                                acc += src[(int64_t)reflect_pop<L>(j, M) * g.slab + rbase + xs];
                                if (wx) acc += src[(int64_t)reflect_pop<L>(j, M | 1) * g.slab + rbase + xs];
                            }
                        }
                    });
                }
            }
            f[j][v] = acc;
        }
    });
}

// The periodic two-phase gather split in two calls, so that a kernel can
// issue the vector loads of two fields before it shuffles either (the same
// loads and halo scalars as gather_two_phase).  REV pulls from x + e_i, the
// adjoint's reverse pull, instead of x - e_i.  gather_late_finish shifts by
// e_x and reads the row-end wrap of the lane holding the row's last node.
template <class L, typename T, int V, bool REV>
__device__ __forceinline__ void gather_early(const T *__restrict__ src, const Geom &g, const RowPos &rpos, int x0,
                                             int lane, T (&f)[L::Q][V], T (&halo)[L::Q])
{
    const int xb = x0 + V * lane;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int sg = REV ? -1 : 1;
        constexpr int ex = sg * L::E[i][0], ey = sg * L::E[i][1], ez = sg * L::E[i][2], ew = sg * L::E[i][3];
        const T *rp = src + (int64_t)i * g.slab + src_row<L::D, ey, ez, ew>(g, rpos) * g.pitch;
        ld_vec(rp + xb, f[i]);
        halo[i] = T(0);
        if constexpr (ex == 1) {
            if (lane == 0) halo[i] = rp[xb == 0 ? g.N0 - 1 : xb - 1];
        } else if constexpr (ex == -1) {
            const int x = xb + V - 1;
            if (lane == 31 && x + 1 < g.N0) halo[i] = rp[x + 1];
        }
    });
}

template <class L, typename T, int V, bool REV>
__device__ __forceinline__ void gather_late_finish(const T *__restrict__ src, const Geom &g, const RowPos &rpos,
                                                   int x0, int lane, T (&f)[L::Q][V], const T (&halo)[L::Q])
{
    const int xb = x0 + V * lane;
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int sg = REV ? -1 : 1;
        constexpr int ex = sg * L::E[i][0], ey = sg * L::E[i][1], ez = sg * L::E[i][2], ew = sg * L::E[i][3];
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
                const T *wp = src + (int64_t)i * g.slab + src_row<L::D, ey, ez, ew>(g, rpos) * g.pitch;
#pragma unroll
                for (int k = 0; k < V; ++k)
                    if (xb + k + 1 == g.N0) f[i][k] = wp[0];
            }
        }
    });
}

// Moments of one node's distributions in the accumulation type of the
// storage (exact int64 sums for fixed point): theta, J_a, P_aa, P_ab.
template <class L, typename A> struct NodeMoments {
    static constexpr int D = L::D, NP = D * (D - 1) / 2 > 0 ? D * (D - 1) / 2 : 1;
    A th, J[D], Paa[D], Pab[NP];
};
template <class L, typename A> __device__ __forceinline__ NodeMoments<L, A> node_moments(const A *f)
{
    constexpr int D = L::D, NP = D * (D - 1) / 2, B0 = 1 + 2 * D;
    NodeMoments<L, A> m;
    m.th = f[0];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        m.Paa[a] = f[1 + a] + f[1 + D + a];
        m.J[a] = f[1 + a] - f[1 + D + a];
        m.th += m.Paa[a];
    }
    static_for<0, NP>([&](auto Pi) {
        constexpr int p = decltype(Pi)::value;
        constexpr int a = pair_a<D>(p), b = pair_b<D>(p);
        const Plane<A> pl = plane(f[B0 + 4 * p], f[B0 + 4 * p + 1], f[B0 + 4 * p + 2], f[B0 + 4 * p + 3]);
        m.th += pl.F;
        m.Paa[a] += pl.F;
        m.Paa[b] += pl.F;
        m.J[a] += pl.Ja;
        m.J[b] += pl.Jb;
        m.Pab[p] = pl.P;
    });
    return m;
}

// Fused multiply-add in the adjoint's own type (fmaf keeps float arithmetic in float).
__device__ __forceinline__ float fma_a(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_a(double a, double b, double c) { return fma(a, b, c); }

template <typename A> __device__ __forceinline__ const Coll<A> &coll_k(const AdjK &K);
template <> __device__ __forceinline__ const Coll<double> &coll_k<double>(const AdjK &K) { return K.k; }
template <> __device__ __forceinline__ const Coll<float> &coll_k<float>(const AdjK &K) { return K.kf; }
template <typename A> __device__ __forceinline__ const Coll<A> &coll_kd(const AdjK &K);
template <> __device__ __forceinline__ const Coll<double> &coll_kd<double>(const AdjK &K) { return K.kd; }
template <> __device__ __forceinline__ const Coll<float> &coll_kd<float>(const AdjK &K) { return K.kdf; }

// One node of the reverse step: l <- K^T l in place (shared sub-sums, as
// in the forward collision); with NU, also returns lambda . (dK/deps) f for
// the node's pre-collision f (stored values fv: f = fv scale + shift).
// A is the adjoint's arithmetic: double, or float for FP32-shifted states.
template <class L, typename T, bool NU, typename A>
__device__ __forceinline__ A adj_node(A *l, const T *fv, const AdjK &K)
{
    constexpr int D = L::D, NP = D * (D - 1) / 2, B0 = 1 + 2 * D;
    const A l0 = l[0];
    A s[D], dd[D], P[NP > 0 ? NP : 1];
    A sax = 0, sdg = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        s[a] = l[1 + a] + l[1 + D + a];
        dd[a] = l[1 + a] - l[1 + D + a];
        sax += s[a];
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const Plane<A> pl = plane(l[B0 + 4 * p], l[B0 + 4 * p + 1], l[B0 + 4 * p + 2], l[B0 + 4 * p + 3]);
        P[p] = pl.P;
        sdg += pl.F;
    }
    A eterm = 0;
    if constexpr (NU) {
        const NodeMoments<L, T> m = node_moments<L, T>(fv);
        // f moments: theta = sum f, P_aa gains sigma theta_ref from the FP32
        // storage shift (w theta_ref has no J or P_ab part)
        A th, Paa[D], J[D], Pab[NP > 0 ? NP : 1];
        if constexpr (std::is_same<T, double>::value) {  // FP64 states: scale 1, no shift
            th = m.th;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                Paa[a] = m.Paa[a];
                J[a] = m.J[a];
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) Pab[p] = m.Pab[p];
        } else if constexpr (std::is_same<A, float>::value && std::is_same<T, float>::value) {
            th = m.th + K.mshift_th_f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                Paa[a] = m.Paa[a] + K.mshift_paa_f;
                J[a] = m.J[a];
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) Pab[p] = m.Pab[p];
        } else {
            th = (A)((double)m.th * K.scale + K.mshift_th);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                Paa[a] = (A)((double)m.Paa[a] * K.scale + K.mshift_paa);
                J[a] = (A)((double)m.J[a] * K.scale);
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) Pab[p] = (A)((double)m.Pab[p] * K.scale);
        }
        const Coll<A> &kd = coll_kd<A>(K);
        eterm = th * fma_a(kd.c0, l0, fma_a(kd.cA, sax, kd.wd * sdg));
#pragma unroll
        for (int a = 0; a < D; ++a) {
            eterm = fma_a(Paa[a], kd.k2 * (s[a] - (A)2 * l0), eterm);
            eterm = fma_a(J[a], kd.k1 * dd[a], eterm);
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) eterm = fma_a(Pab[p], kd.k3 * P[p], eterm);
    }
    const Coll<A> &k = coll_k<A>(K);
    const A Lt = fma_a(k.c0, l0, fma_a(k.cA, sax, k.wd * sdg));
    A LP[D], LJ[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        LP[a] = k.k2 * (s[a] - (A)2 * l0);
        LJ[a] = k.k1 * dd[a];
    }
    l[0] = Lt;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const A base = Lt + LP[a];
        l[1 + a] = base + LJ[a];
        l[1 + D + a] = base - LJ[a];
    }
    static_for<0, NP>([&](auto Pi) {
        constexpr int p = decltype(Pi)::value;
        constexpr int a = pair_a<D>(p), b = pair_b<D>(p);
        const A X = Lt + (LP[a] + LP[b]);
        const A U = LJ[a] + LJ[b], W = LJ[a] - LJ[b];
        const A lab = k.k3 * P[p];
        const A Xp = X + lab, Xm = X - lab;
        l[B0 + 4 * p] = Xp + U;      // (+1, +1)
        l[B0 + 4 * p + 1] = Xm - W;  // (-1, +1)
        l[B0 + 4 * p + 2] = Xp - U;  // (-1, -1)
        l[B0 + 4 * p + 3] = Xm + W;  // (+1, -1)
    });
    return eterm;
}

// The eps-term of fixed-point nodes, before its last conversions: the FP64
// part theta * (c0' l0 + cA' sum_a + wd' sum_diag), and the exact 128-bit
// dot products S2 = sum P_aa s2_a, S1 = sum J_a dd_a, S3 = sum P_ab P_p of
// the state's integer moments with the integer lambda channels.  A lane sums
// its nodes' S (each below 6 * 2^122 in magnitude for channels below 2^59 and
// moments below 2^63, so two nodes' sum stays far inside 2^127) and converts
// each sum once: eps-term = d + k2' S2 + k1' S1 + k3' S3.
struct EpsFx {
    double d = 0.0;
    __int128 S2 = 0, S1 = 0, S3 = 0;
};

// The node update of the fixed-point reverse pass (64-bit fixed-point states):
// K^T from exact integer channel sums and rounded 64x62-bit products; with
// NU, the eps-term lambda . (dK/deps) f as EpsFx (the int64 channel and
// moment values of its FP64 part by the hardware conversion, which keeps the
// FP64 and integer pipes in balance).  ORs into `rng` the high words of the
// outputs plus 2^27: an output is inside |v| < 2^59 (the fields start below
// 2^56) exactly when that sum stays below 2^28.
template <class L, bool NU>
__device__ __forceinline__ void adj_node_fx(long long *l, const long long *fv, const AdjK &K, unsigned &rng, EpsFx &ep)
{
    constexpr int D = L::D, NP = D * (D - 1) / 2, B0 = 1 + 2 * D;
    const long long l0 = l[0];
    long long s2[D], dd[D], P[NP > 0 ? NP : 1];  // s2 = l_{+a} + l_{-a} - 2 l0
    long long sax = 0, sdg = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const long long sa = l[1 + a] + l[1 + D + a];
        sax += sa;
        s2[a] = sa - 2 * l0;
        dd[a] = l[1 + a] - l[1 + D + a];
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const Plane<long long> pl = plane(l[B0 + 4 * p], l[B0 + 4 * p + 1], l[B0 + 4 * p + 2], l[B0 + 4 * p + 3]);
        P[p] = pl.P;
        sdg += pl.F;
    }
    if constexpr (NU) {
        const NodeMoments<L, long long> m = node_moments<L, long long>(fv);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            ep.S2 += (__int128)m.Paa[a] * s2[a];
            ep.S1 += (__int128)m.J[a] * dd[a];
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) ep.S3 += (__int128)m.Pab[p] * P[p];
        const Coll<double> &kd = K.kdx;
        const double lt = fma(kd.c0, (double)l0, fma(kd.cA, (double)sax, kd.wd * (double)sdg));
        ep.d = fma((double)m.th, lt, ep.d);
    }
    // the rest channel: one rounding of the exact sum of its three products
    const __int128 lts = (__int128)l0 * K.c0k + (__int128)sax * K.cAk + (__int128)sdg * K.wdk;
    const long long Lt = (long long)((lts + ((__int128)1 << (kFxCoefBits - 1))) >> kFxCoefBits);
    long long LP[D], LJ[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        LP[a] = mulfx(s2[a], K.k2k);
        LJ[a] = mulfx(dd[a], K.k1k);
    }
    l[0] = Lt;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const long long base = Lt + LP[a];
        l[1 + a] = base + LJ[a];
        l[1 + D + a] = base - LJ[a];
    }
    static_for<0, NP>([&](auto Pi) {
        constexpr int p = decltype(Pi)::value;
        constexpr int a = pair_a<D>(p), b = pair_b<D>(p);
        const long long X = Lt + (LP[a] + LP[b]);
        const long long U = LJ[a] + LJ[b], W = LJ[a] - LJ[b];
        const long long lab = mulfx(P[p], K.k3k);
        const long long Xp = X + lab, Xm = X - lab;
        l[B0 + 4 * p] = Xp + U;      // (+1, +1)
        l[B0 + 4 * p + 1] = Xm - W;  // (-1, +1)
        l[B0 + 4 * p + 2] = Xp - U;  // (-1, -1)
        l[B0 + 4 * p + 3] = Xm + W;  // (+1, -1)
    });
    // next step's channel sums (<= 12 terms below 2^59) stay below 2^63
#pragma unroll
    for (int i = 0; i < L::Q; ++i) rng |= (unsigned)((unsigned long long)l[i] >> 32) + (1u << 27);
}

// The integer -> FP64 conversions of the fixed-point eps-term, for their self-test.
__global__ void int_to_f64_selftest_kernel(const long long *__restrict__ hi, const unsigned long long *__restrict__ lo,
                                           int64_t n, double *__restrict__ out128, double *__restrict__ out64)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const __int128 v = (__int128)(((unsigned __int128)(unsigned long long)hi[i] << 64) | lo[i]);
        out128[i] = i128_to_f64_rn(v);
        out64[i] = i64_to_f64_rn((long long)lo[i]);
    }
}

// Sum type of a lane's eps-terms: the adjoint's own type, FP64 for fixed point.
template <typename A> using EpsAcc = typename std::conditional<std::is_same<A, long long>::value, double, A>::type;

// FP64 seed values -> fixed point round(v * 2^G).
__global__ void to_fixed_kernel(const double *__restrict__ src, long long *__restrict__ dst, int64_t n,
                                double scale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __double2ll_rn(src[i] * scale);
}

template <typename A> __device__ __forceinline__ A warp_sum(A v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// phi_T = dL/df_T through u_a = ucoef J_a / theta and, where dLdth is given,
// theta = sum_k f_k (d theta / d f_k = 1); eps-term of the recovery (theta has
// no explicit eps dependence).  dLdu or dLdth may be NULL (not both).
template <class L, typename T, typename A, bool MIR = false>
__global__ void __launch_bounds__(kSweepThreads) adj_seed_kernel(const T *__restrict__ P, Geom g, AdjK K,
                                                                 const double *__restrict__ dLdu,
                                                                 const double *__restrict__ dLdth,
                                                                 A *__restrict__ phi, double *__restrict__ slot)
{
    constexpr int V = 2;
    const int lane = threadIdx.x & 31;
    const int64_t seg = (int64_t)blockIdx.x * (kSweepThreads / 32) + (threadIdx.x >> 5);
    if (seg >= g.nseg) return;
    const int64_t row = seg / g.seg_per_row;
    const int x0 = (int)(seg - row * g.seg_per_row) * (32 * V);
    T f[L::Q][V];
    gather<L, T, V, MIR>(P, g, row, x0, lane, f);
    const int64_t nodes = (int64_t)g.N0 * g.rows;
    double out[L::Q][V];
    double acc = 0.0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int x = x0 + V * lane + v;
        double th = 0.0, J[3] = {0.0, 0.0, 0.0};
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const double fv = to_f(f[i][v], K.scale) + K.shift[i];
            th += fv;
            static_for<0, L::D>([&](auto Ad) {
                constexpr int a = decltype(Ad)::value;
                constexpr int e = L::E[i][a];
                if constexpr (e != 0) J[a] += e * fv;
            });
        });
        double gu[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0}, gt = 0.0;
        if (x < g.N0) {
            const int64_t node = row * g.N0 + x;
            if (dLdu) {
#pragma unroll
                for (int a = 0; a < L::D; ++a) {
                    gu[a] = dLdu[a * nodes + node];
                    u[a] = K.ucoef * J[a] / th;
                    acc += gu[a] * K.ducoef * J[a] / th;
                }
            }
            if (dLdth) gt = dLdth[node];
        }
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            double s = 0.0;
            static_for<0, L::D>([&](auto Ad) {
                constexpr int a = decltype(Ad)::value;
                constexpr int e = L::E[i][a];
                s += gu[a] * ((double)e * K.ucoef - u[a]);
            });
            out[i][v] = (x < g.N0) ? s / th + gt : 0.0;
        });
    }
    if (x0 + V * lane < g.pitch) {  // lanes beyond the row only loaded
        A *dp = phi + row * g.pitch + x0 + V * lane;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            A o[V];
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = (A)out[i][v];
            st_vec(dp + (int64_t)i * g.slab, o);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) slot[seg] += acc;
}

// Threads per block of the reverse step: 128 (FP32: its early-issued gathers
// need 72 registers, and at 256 threads a 512^2 step would no longer fit one
// wave; FP64: at about 90 registers 128-thread blocks keep 20 warps per SM
// resident instead of 16; fixed point: measured 20.9 against 21.7 us per
// 512^2 step with 256).
template <typename A> __host__ __device__ constexpr int adj_threads()
{
    return 128;
}

// One reverse step: phi_out = K^T lambda(phi_in); eps-term if NU.
template <class L, typename T, bool NU, typename A, bool MIR = false>
__global__ void __launch_bounds__(adj_threads<A>()) adj_step_kernel(const A *__restrict__ phi_in,
                                                                 const T *__restrict__ Pn, A *__restrict__ phi_out,
                                                                 Geom g, AdjK K, double *__restrict__ slot,
                                                                 int *__restrict__ flag)
{
    constexpr int V = 2;
    const int lane = threadIdx.x & 31;
    const int64_t seg = (int64_t)blockIdx.x * (adj_threads<A>() / 32) + (threadIdx.x >> 5);
    if (seg >= g.nseg) return;
    const int64_t row = seg / g.seg_per_row;
    const int x0 = (int)(seg - row * g.seg_per_row) * (32 * V);
    A lam[L::Q][V];
    T f[L::Q][V];
    if constexpr (!MIR && NU && std::is_same<A, float>::value) {
        // FP32: the vector loads of both fields in flight before either is shuffled
        const RowPos rpos = row_pos<L::D>(g, row);
        A hl[L::Q];
        T hf[L::Q];
        gather_early<L, A, V, true>(phi_in, g, rpos, x0, lane, lam, hl);
        gather_early<L, T, V, false>(Pn, g, rpos, x0, lane, f, hf);
        gather_late_finish<L, A, V, true>(phi_in, g, rpos, x0, lane, lam, hl);
        gather_late_finish<L, T, V, false>(Pn, g, rpos, x0, lane, f, hf);
    } else {
        if constexpr (MIR)
            gather_rev_walls<L, A>(phi_in, g, row, x0, lane, lam);
        else
            gather_rev<L, A>(phi_in, g, row, x0, lane, lam);
        if constexpr (NU) gather<L, T, V, MIR>(Pn, g, row, x0, lane, f);
    }
    EpsAcc<A> acc = 0;  // this lane's dL/deps terms
    bool range = false;
    EpsFx ep;  // fixed point: the lane's eps-term sums, converted once below
#pragma unroll
    for (int v = 0; v < V; ++v) {
        A l[L::Q];
        T fv[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            l[i] = lam[i][v];
            if constexpr (NU) fv[i] = f[i][v];
        }
        // lanes past the row end hold values of the allocation's slack (never
        // initialised): only the grid's own nodes may set the flag or add terms
        const bool own = x0 + V * lane + v < g.N0;
        if constexpr (std::is_same<A, long long>::value) {
            unsigned rng = 0u;
            EpsFx e;
            adj_node_fx<L, NU>(l, fv, K, rng, e);
            if (own) {
                range |= rng >= (1u << 28);
                ep.d += e.d;
                ep.S2 += e.S2;
                ep.S1 += e.S1;
                ep.S3 += e.S3;
            }
        } else {
            const EpsAcc<A> e = adj_node<L, T, NU, A>(l, fv, K);
            if (NU && own) acc += e;
        }
#pragma unroll
        for (int i = 0; i < L::Q; ++i) lam[i][v] = l[i];
    }
    if constexpr (std::is_same<A, long long>::value && NU) {
        const Coll<double> &kd = K.kdx;
        acc = ep.d + fma(kd.k2, i128_to_f64_rn(ep.S2), fma(kd.k1, i128_to_f64_rn(ep.S1), kd.k3 * i128_to_f64_rn(ep.S3)));
    }
    if (x0 + V * lane < g.pitch) {  // lanes beyond the row only loaded
        A *dp = phi_out + row * g.pitch + x0 + V * lane;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) st_vec(dp + (int64_t)i * g.slab, lam[i]);
    }
    if constexpr (std::is_same<A, long long>::value) {
        if (range) atomicOr(flag, 1);
    }
    if constexpr (NU) {
        // one writer per slot per launch, launches in stream order: the
        // reduction (no return value, so the warp does not wait) is deterministic
        acc = warp_sum(acc);
        if (lane == 0) atomicAdd(slot + seg, (double)acc);
    }
}

// Adjoint of the initialisation f_i = w_i theta0 - sum_a A_ia d_a theta0:
// dtheta0 = sum_i w_i phi_i, h_a = -sum_i A_ia phi_i (fed to G^T), and the
// eps-term sum_i phi_i (w_i' theta0 - sum_a A'_ia d_a theta0).
template <class L, typename A>
__global__ void adj_init_kernel(const A *__restrict__ phi, Geom g, AdjK K, const double *__restrict__ th0,
                                const double *__restrict__ grad, double *__restrict__ dth0,
                                double *__restrict__ h, double *__restrict__ slot)
{
    const int64_t nodes = (int64_t)g.N0 * g.rows;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (n < nodes) {
        const int x = (int)(n % g.N0);
        const int64_t rw = n / g.N0;
        const A *p = phi + rw * g.pitch + x;
        const double t0 = th0[n];
        // on a wall node the initialisation takes the wall-normal gradient as
        // zero: no dependence on it, no term through it
        const int cc[3] = {x, (int)(rw % g.N1), (int)(rw / g.N1)};
        const int nn[3] = {g.N0, g.N1, g.N2};
        bool onwall[3] = {false, false, false};
        double gr[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            onwall[a] = ((g.mirror >> a) & 1u) && (cc[a] == 0 || cc[a] == nn[a] - 1);
            gr[a] = onwall[a] ? 0.0 : grad[a * nodes + n];
        }
        double s = 0.0, hh[3] = {0.0, 0.0, 0.0};
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ex = L::E[i][0], ey = L::E[i][1], ez = L::E[i][2];
            constexpr int nz = (ex != 0) + (ey != 0) + (ez != 0);
            const double ph = std::is_same<A, long long>::value ? (double)p[(int64_t)i * g.slab] * K.aunit
                                                               : (double)p[(int64_t)i * g.slab];
            s = fma(K.w[i], ph, s);
            double dfi = K.dw[i] * t0;
            if constexpr (nz == 1) {
                constexpr int a = (ex != 0) ? 0 : ((ey != 0) ? 1 : 2);
                constexpr int sg = (ex != 0) ? ex : ((ey != 0) ? ey : ez);
                hh[a] -= sg * K.iax * ph;
                dfi -= sg * K.diax * gr[a];
            } else if constexpr (nz == 2) {
                if constexpr (ex != 0) hh[0] -= ex * K.idg * ph;
                if constexpr (ey != 0) hh[1] -= ey * K.idg * ph;
                if constexpr (ez != 0) hh[2] -= ez * K.idg * ph;
                dfi -= K.didg * (ex * gr[0] + ey * gr[1] + ez * gr[2]);
            }
            acc = fma(ph, dfi, acc);
        });
        dth0[n] = s;
#pragma unroll
        for (int a = 0; a < L::D; ++a) h[a * nodes + n] = onwall[a] ? 0.0 : hh[a];
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) slot[n >> 5] += acc;
}

// dth0 += G^T h, with (G^T h)(x) = sum_a sum_k cof_k h_a(x - off_k e_a) / (12 dx)
// on periodic axes.  On an axis with walls the forward difference reads
// theta at the even reflection of x + off_k, so node y also collects the
// terms whose reflected read lands on it: from x = -y - off_k (read beyond
// the first wall) and x = 2(n - 1) - y - off_k (beyond the last).
__global__ void adj_fd4t_kernel(const double *__restrict__ h, double *__restrict__ dth0, int d, int N0, int N1,
                                int N2, unsigned mirror, double inv12dx)
{
    const int64_t nodes = (int64_t)N0 * N1 * N2;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
    const int x = (int)(n % N0);
    const int64_t rw = n / N0;
    const int y = (int)(rw % N1);
    const int z = (int)(rw / N1);
    const int nn[3] = {N0, N1, N2};
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
        const int off[4] = {2, 1, -1, -2};
        const double cof[4] = {-1.0, 8.0, -8.0, 1.0};
        const int ya = (a == 0) ? x : ((a == 1) ? y : z), na = nn[a];
        for (int k = 0; k < 4; ++k) {
            int xs[3], cnt = 0;
            if ((mirror >> a) & 1u) {
                const int direct = ya - off[k];
                if (direct >= 0 && direct < na) xs[cnt++] = direct;
                const int lo = -ya - off[k];  // x + off_k = -y < 0 reflects onto y
                if (ya > 0 && lo >= 0 && lo < na && lo + off[k] < 0) xs[cnt++] = lo;
                const int hi = 2 * (na - 1) - ya - off[k];  // x + off_k > n - 1 reflects onto y
                if (ya < na - 1 && hi >= 0 && hi < na && hi + off[k] > na - 1) xs[cnt++] = hi;
            } else {
                xs[cnt++] = ((ya - off[k]) % na + na) % na;
            }
            for (int m = 0; m < cnt; ++m) {
                int c[3] = {x, y, z};
                c[a] = xs[m];
                s += cof[k] * h[a * nodes + ((int64_t)c[2] * N1 + c[1]) * N0 + c[0]];
            }
        }
    }
    dth0[n] += s * inv12dx;
}

// Fixed-order sum of n doubles into out[0] (one block).
__global__ void __launch_bounds__(256) sum_slots_kernel(const double *__restrict__ a, int64_t n,
                                                        const double *__restrict__ b, int64_t nb,
                                                        double *__restrict__ out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) s += a[i];
    for (int64_t i = threadIdx.x; i < nb; i += 256) s += b[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

}  // namespace lbk

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct lb_adj {
    lb_ctx *ctx = nullptr;
    lbk::Geom ag{};  // the state's rows cut into 64-node segments (2 per lane)
    int64_t T = 0, C = 0, nck = 0;
    bool want_nu = false;
    size_t state_bytes = 0;
    std::vector<void *> ck;      // checkpoints P_{kC}
    std::vector<void *> seg[2];  // recomputed segments P_{kC + m}: segment k in seg[k & 1] (seg[0] alone if one)
    int nseg_buf = 1;            // 2 when the next segment is recomputed while the current one is reversed
    int64_t seg_loaded[2] = {-1, -1};
    void *phi[2] = {nullptr, nullptr};  // adjoint fields: float (FP32s), int64 fixed point (fx), else double
    bool fx = false;                     // fixed-point reverse pass (64-bit fixed-point states)
    int *dflag = nullptr;                // fixed-point range flag
    int pcur = 0;
    double *th0 = nullptr, *grad = nullptr, *h = nullptr;
    double *slot_step = nullptr, *slot_init = nullptr, *dsum = nullptr;
    int64_t nslot_init = 0;
    int64_t done = 0;  // reverse steps completed
    bool forward_done = false, seeded = false;
    lbk::AdjK K{};
    size_t bytes = 0;
    // Recorded graphs.  fgraph[p]: C forward sweeps from buffer p (valid for
    // the walls they were recorded with).  rgraph[p][b][pre]: one whole
    // reverse segment, C reverse steps from adjoint buffer p over the segment
    // held in seg[b], and with pre = 1 beside them, on a second branch, the
    // C - 1 recompute sweeps of the previous segment into seg[b ^ 1] (valid
    // for the constants K and walls they were recorded with).
    cudaGraphExec_t fgraph[2] = {nullptr, nullptr};
    uint64_t fgen[2] = {0, 0};  // the context's generation (walls, viscosity) each was recorded in
    uint64_t fwd_gen = 0;       // the context's generation at the last forward pass
    cudaGraphExec_t rgraph[2][2][2] = {};
    lbk::AdjK rK[2][2][2]{};
    unsigned rmirror[2][2][2] = {};
};

namespace {

lb_status afail(lb_adj *a, lb_status s, const std::string &m)
{
    if (a && a->ctx) a->ctx->err = m;
    return s;
}

lb_status acuda(lb_adj *a, cudaError_t e, const char *where)
{
    return afail(a, e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

void free_adj(lb_adj *a)
{
    if (!a) return;
    for (void *p : a->ck) cudaFree(p);
    for (auto &sb : a->seg)
        for (void *p : sb) cudaFree(p);
    cudaFree(a->phi[0]);
    cudaFree(a->phi[1]);
    cudaFree(a->th0);
    cudaFree(a->grad);
    cudaFree(a->h);
    cudaFree(a->slot_step);
    cudaFree(a->slot_init);
    cudaFree(a->dsum);
    cudaFree(a->dflag);
    for (int p = 0; p < 2; ++p) {
        if (a->fgraph[p]) cudaGraphExecDestroy(a->fgraph[p]);
        for (auto &gb : a->rgraph[p])
            for (cudaGraphExec_t g : gb)
                if (g) cudaGraphExecDestroy(g);
    }
    delete a;
}

// Record into *out the launches `body` makes on the context's stream (swapped
// for a private capturing stream meanwhile).
template <class F> cudaError_t record_graph(lb_ctx *c, cudaGraphExec_t *out, F &&body)
{
    if (*out) {
        cudaGraphExecDestroy(*out);
        *out = nullptr;
    }
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaStream_t user = c->stream;
    c->stream = cs;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = body();
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return e;
}

bool stream_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return true;
    return cap != cudaStreamCaptureStatusNone;
}

// Collision, recovery and initialisation constants and their eps-derivatives
// (Theorem 2, Eq. (Bur-Sol), differentiated in eps).
void make_adjk(lb_adj *a)
{
    const lb_ctx &c = *a->ctx;
    const int d = c.d;
    const double eps = c.eps, A = 6.0 * eps + 1.0, B = 6.0 * eps + 3.0;
    double ds1 = 0, ds2x = 0, ds22 = 0, dw1 = 0, dwd = 0;
    if (c.paper) {
        ds1 = -12.0 / (A * A);
        ds2x = 24.0 / (A * A) - 288.0 * eps / (A * A * A);
        if (d > 1) {
            ds22 = -24.0 / (B * B);
            dw1 = -(d - 1) / 3.0;
            dwd = 1.0 / 6.0;
        }
    }
    const double sigma = c.sigma, dsigma = 2.0 * dw1 + 4.0 * (d - 1) * dwd;
    const double wd = (d > 1) ? c.wd : 0.0;
    lbk::AdjK &K = a->K;
    K.k = lbk::make_coll<double>(c);
    K.kd.k1 = -ds1 / 2.0;
    K.kd.k2 = -ds2x / 2.0;
    K.kd.k3 = -ds22 / 4.0;
    K.kd.c0 = -d * (ds2x * sigma + c.s2x * dsigma) + 2.0 * d * (d - 1) * dwd;
    K.kd.cA = (ds2x * sigma + c.s2x * dsigma) / 2.0 - 2.0 * (d - 1) * dwd;
    K.kd.wd = dwd;
    K.kf = lbk::make_coll<float>(c);
    const auto fxk = [](double v) { return llrint(ldexp(v, lbk::kFxCoefBits)); };
    K.c0k = fxk(K.k.c0);
    K.cAk = fxk(K.k.cA);
    K.wdk = fxk(K.k.wd);
    K.k1k = fxk(K.k.k1);
    K.k2k = fxk(K.k.k2);
    K.k3k = fxk(K.k.k3);
    K.aunit = 1.0;
    K.kdx = K.kd;
    K.kdf = {(float)K.kd.k1, (float)K.kd.k2, (float)K.kd.k3, (float)K.kd.c0, (float)K.kd.cA, (float)K.kd.wd};
    const int q = c.q;
    double w[lbk::kAdjQ], dw[lbk::kAdjQ];
    w[0] = c.w0;
    dw[0] = -2.0 * d * dw1 - 2.0 * d * (d - 1) * dwd;
    for (int i = 1; i < q; ++i) {
        w[i] = (i <= 2 * d) ? c.w1 : wd;
        dw[i] = (i <= 2 * d) ? dw1 : dwd;
    }
    for (int i = 0; i < lbk::kAdjQ; ++i) {
        K.w[i] = i < q ? w[i] : 0.0;
        K.dw[i] = i < q ? dw[i] : 0.0;
        K.shift[i] = 0.0;
    }
    K.scale = (c.precision == LB_FX64) ? ldexp(1.0, -c.fx_bits) : 1.0;
    K.mshift_th = K.mshift_paa = 0.0;
    if (c.precision == LB_FP32_SHIFTED) {  // stored f - w theta_ref
        for (int i = 0; i < q; ++i) K.shift[i] = w[i] * c.theta_ref;
        K.mshift_th = c.theta_ref;
        K.mshift_paa = sigma * c.theta_ref;
    }
    K.mshift_th_f = (float)K.mshift_th;
    K.mshift_paa_f = (float)K.mshift_paa;
    K.ucoef = (2.0 - c.s1) * c.c;
    K.ducoef = -ds1 * c.c;
    K.iax = 0.5 * c.dx * (sigma / c.s1 - 4.0 * (d - 1) * wd);
    K.diax = 0.5 * c.dx * (dsigma / c.s1 - sigma * ds1 / (c.s1 * c.s1) - 4.0 * (d - 1) * dwd);
    K.idg = wd * c.dx;
    K.didg = dwd * c.dx;
    K.inv12dx = 1.0 / (12.0 * c.dx);
}

int64_t sweep_blocks(const lbk::Geom &g) { return (g.nseg + lbk::kSweepThreads / 32 - 1) / (lbk::kSweepThreads / 32); }

// The adjoint's arithmetic for a storage type: float for FP32-shifted states
// (whose forward map is only FP32-accurate), double otherwise; fixed-point
// states use the integer reverse pass (a->fx) when its constants fit.
template <typename T> using AdjT = typename std::conditional<std::is_same<T, float>::value, float, double>::type;

// Constants of the fixed-point reverse pass once the adjoint scale 2^G is known.
void set_fx_scale(lb_adj *a, int G)
{
    lbk::AdjK &K = a->K;
    K.aunit = ldexp(1.0, -G);
    const int sh = -(a->ctx->fx_bits + G);
    K.kdx = {ldexp(K.kd.k1, sh), ldexp(K.kd.k2, sh), ldexp(K.kd.k3, sh),
             ldexp(K.kd.c0, sh), ldexp(K.kd.cA, sh), ldexp(K.kd.wd, sh)};
}

template <class L, typename T> cudaError_t seed_t(lb_adj *a, const double *dLdu, const double *dLdth)
{
    lb_ctx *c = a->ctx;
    const unsigned nb = (unsigned)sweep_blocks(a->ag);
    if constexpr (std::is_same<T, long long>::value) {
        if (a->fx) {
            // FP64 seed into the other field, then round(phi 2^G) with max|phi| 2^G < 2^56:
            // seven bits of headroom for the channel sums and the (measured, < 1.3x) growth
            double *tmp = (double *)a->phi[a->pcur ^ 1];
            if (a->ag.mirror)
                lbk::adj_seed_kernel<L, T, double, true><<<nb, lbk::kSweepThreads, 0, c->stream>>>(
                    (const T *)c->f[c->cur], a->ag, a->K, dLdu, dLdth, tmp, a->slot_step);
            else
                lbk::adj_seed_kernel<L, T, double><<<nb, lbk::kSweepThreads, 0, c->stream>>>(
                    (const T *)c->f[c->cur], a->ag, a->K, dLdu, dLdth, tmp, a->slot_step);
            cudaError_t e = cudaGetLastError();
            const int64_t n = (int64_t)c->q * a->ag.slab;
            double mx = 0.0;
            if (e == cudaSuccess) e = lbk::launch_maxabs(c, tmp, n, c->dout);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&mx, c->dout, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return e;
            int ex = 0;
            if (mx > 0.0) frexp(mx, &ex);
            const int G = 56 - ex;
            set_fx_scale(a, G);
            lbk::to_fixed_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, c->stream>>>(
                tmp, (long long *)a->phi[a->pcur], n, ldexp(1.0, G));
            return cudaGetLastError();
        }
    }
    using A = AdjT<T>;
    if (a->ag.mirror)
        lbk::adj_seed_kernel<L, T, A, true><<<nb, lbk::kSweepThreads, 0, c->stream>>>(
            (const T *)c->f[c->cur], a->ag, a->K, dLdu, dLdth, (A *)a->phi[a->pcur], a->slot_step);
    else
        lbk::adj_seed_kernel<L, T, A><<<nb, lbk::kSweepThreads, 0, c->stream>>>(
            (const T *)c->f[c->cur], a->ag, a->K, dLdu, dLdth, (A *)a->phi[a->pcur], a->slot_step);
    return cudaGetLastError();
}

template <class L, typename T, typename A, bool MIR> cudaError_t step_m(lb_adj *a, const void *Pn)
{
    lb_ctx *c = a->ctx;
    constexpr int TH = lbk::adj_threads<A>();
    const unsigned nb = (unsigned)((a->ag.nseg + TH / 32 - 1) / (TH / 32));
    const A *in = (const A *)a->phi[a->pcur];
    A *out = (A *)a->phi[a->pcur ^ 1];
    if (a->want_nu)
        lbk::adj_step_kernel<L, T, true, A, MIR><<<nb, TH, 0, c->stream>>>(
            in, (const T *)Pn, out, a->ag, a->K, a->slot_step, a->dflag);
    else
        lbk::adj_step_kernel<L, T, false, A, MIR><<<nb, TH, 0, c->stream>>>(
            in, (const T *)Pn, out, a->ag, a->K, a->slot_step, a->dflag);
    return cudaGetLastError();
}

template <class L, typename T, typename A> cudaError_t step_a(lb_adj *a, const void *Pn)
{
    return a->ag.mirror ? step_m<L, T, A, true>(a, Pn) : step_m<L, T, A, false>(a, Pn);
}

template <class L, typename T> cudaError_t step_t(lb_adj *a, const void *Pn)
{
    if constexpr (std::is_same<T, long long>::value) {
        if (a->fx) return step_a<L, T, long long>(a, Pn);
    }
    return step_a<L, T, AdjT<T>>(a, Pn);
}

template <class L, typename A> cudaError_t init_a(lb_adj *a, double *dth0)
{
    lb_ctx *c = a->ctx;
    const unsigned nb = (unsigned)((c->nodes + 255) / 256);
    lbk::adj_init_kernel<L, A><<<nb, 256, 0, c->stream>>>((const A *)a->phi[a->pcur], c->geom, a->K, a->th0, a->grad,
                                                          dth0, a->h, a->slot_init);
    return cudaGetLastError();
}

template <class L> cudaError_t init_t(lb_adj *a, double *dth0)
{
    lb_ctx *c = a->ctx;
    const unsigned nb = (unsigned)((c->nodes + 255) / 256);
    cudaError_t e;
    if (c->precision == LB_FP32_SHIFTED)
        e = init_a<L, float>(a, dth0);
    else if (a->fx)
        e = init_a<L, long long>(a, dth0);
    else
        e = init_a<L, double>(a, dth0);
    if (e != cudaSuccess) return e;
    lbk::adj_fd4t_kernel<<<nb, 256, 0, c->stream>>>(a->h, dth0, c->d, (int)c->N[0], (int)c->N[1], (int)c->N[2],
                                                    c->geom.mirror, a->K.inv12dx);
    return cudaGetLastError();
}

template <class L> cudaError_t seed_l(lb_adj *a, const double *dLdu, const double *dLdth)
{
    switch (a->ctx->precision) {
    case LB_FX64: return seed_t<L, long long>(a, dLdu, dLdth);
    case LB_FP32_SHIFTED: return seed_t<L, float>(a, dLdu, dLdth);
    default: return seed_t<L, double>(a, dLdu, dLdth);
    }
}

cudaError_t do_seed(lb_adj *a, const double *dLdu, const double *dLdth)
{
    switch (a->ctx->d) {
    case 1: return seed_l<lbk::D1Q3>(a, dLdu, dLdth);
    case 2: return seed_l<lbk::D2Q9>(a, dLdu, dLdth);
    default: return seed_l<lbk::D3Q19>(a, dLdu, dLdth);
    }
}

template <class L> cudaError_t step_l(lb_adj *a, const void *Pn)
{
    switch (a->ctx->precision) {
    case LB_FX64: return step_t<L, long long>(a, Pn);
    case LB_FP32_SHIFTED: return step_t<L, float>(a, Pn);
    default: return step_t<L, double>(a, Pn);
    }
}

cudaError_t do_step(lb_adj *a, const void *Pn)
{
    switch (a->ctx->d) {
    case 1: return step_l<lbk::D1Q3>(a, Pn);
    case 2: return step_l<lbk::D2Q9>(a, Pn);
    default: return step_l<lbk::D3Q19>(a, Pn);
    }
}

cudaError_t do_init(lb_adj *a, double *dth0)
{
    switch (a->ctx->d) {
    case 1: return init_t<lbk::D1Q3>(a, dth0);
    case 2: return init_t<lbk::D2Q9>(a, dth0);
    default: return init_t<lbk::D3Q19>(a, dth0);
    }
}

// The segment buffer that holds (or will hold) checkpoint segment k.
int seg_buf(const lb_adj *a, int64_t k) { return a->nseg_buf == 2 ? (int)(k & 1) : 0; }

// Recompute checkpoint segment k into its buffer, on the context's stream.
cudaError_t load_segment(lb_adj *a, int64_t k)
{
    lb_ctx *c = a->ctx;
    const int b = seg_buf(a, k);
    std::vector<void *> &sg = a->seg[b];
    cudaError_t e = cudaMemcpyAsync(sg[0], a->ck[k], a->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
    const int64_t len = std::min<int64_t>(a->C, a->T - k * a->C);
    for (int64_t m = 1; m < len; ++m)
        if ((e = lbk::launch_sweep(c, sg[m - 1], sg[m])) != cudaSuccess) return e;
    a->seg_loaded[b] = k;
    return cudaSuccess;
}

// Make P_n available (n < T): checkpoint segment k = n / C recomputed into its buffer.
cudaError_t state_at(lb_adj *a, int64_t n, const void **out)
{
    const int64_t k = n / a->C;
    const int b = seg_buf(a, k);
    if (a->seg_loaded[b] != k) {
        cudaError_t e = load_segment(a, k);
        if (e != cudaSuccess) return e;
    }
    *out = a->seg[b][n - k * a->C];
    return cudaSuccess;
}

}  // namespace

extern "C" {

lb_status lb_adjoint_create(lb_ctx *ctx, int64_t T, int64_t C, int want_nu, lb_adj **out)
{
    lbk::NvtxRange nvtx_range("lb_adjoint_create");
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (!ctx || T < 1) return LB_EINVAL;
    if (ctx->d > 3) {
        ctx->err = "lb_adjoint_create: the adjoint supports d = 1, 2, 3";
        return LB_EINVAL;
    }
    if (want_nu && !ctx->paper) {
        ctx->err = "lb_adjoint_create: dL/dnu needs the paper's relaxation set";
        return LB_EINVAL;
    }
    if (C == 0) C = (int64_t)ceil(sqrt((double)T));
    if (C < 1 || C > T) {
        ctx->err = "lb_adjoint_create: checkpoint interval out of range";
        return LB_EINVAL;
    }
    lb_adj *a = new (std::nothrow) lb_adj();
    if (!a) return LB_ENOMEM;
    a->ctx = ctx;
    a->ag = ctx->geom;  // 64-node segments: two values per lane for every storage type
    a->ag.seg_per_row = (ctx->geom.pitch + 63) / 64;
    a->ag.nseg = ctx->geom.rows * a->ag.seg_per_row;
    a->T = T;
    a->C = C;
    a->want_nu = want_nu != 0;
    {
        // The integer reverse pass holds the constants with 62 fraction bits
        // (each inside (-2, 2)) and keeps every field below 2^59 (checked per
        // store).  An output of K^T is then bounded by
        // (|c0| + 2d|cA| + 4P|wd| + 8|k2| + 4|k1| + 4|k3|) 2^59, P = d(d-1)/2
        // planes, which must stay below 2^63; otherwise the pass runs in FP64.
        const lbk::Coll<double> kc = lbk::make_coll<double>(*ctx);
        const double d = ctx->d, planes = d * (d - 1) / 2;
        const double bound = fabs(kc.c0) + 2 * d * fabs(kc.cA) + 4 * planes * fabs(kc.wd) + 8 * fabs(kc.k2) +
                             4 * fabs(kc.k1) + 4 * fabs(kc.k3);
        const double lim = 1.999;
        a->fx = ctx->precision == LB_FX64 && bound < 15.0 && fabs(kc.c0) < lim && fabs(kc.cA) < lim &&
                fabs(kc.wd) < lim && fabs(kc.k1) < lim && fabs(kc.k2) < lim && fabs(kc.k3) < lim;
    }
    a->state_bytes = (size_t)ctx->q * ctx->geom.slab * ctx->elem;
    cudaError_t e = cudaSuccess;
    const size_t aelem = (ctx->precision == LB_FP32_SHIFTED) ? sizeof(float) : sizeof(double);
    const size_t pbytes = ((size_t)ctx->q * ctx->geom.slab + lbk::kSlackElems) * aelem;
    const size_t sbytes = a->state_bytes + lbk::kSlackElems * ctx->elem;  // allocation incl. slack
    if (a->want_nu) {
        a->nck = (T + C - 1) / C;
        a->nseg_buf = 1;  // a second segment buffer is added below when the device has room for it
        a->ck.assign(a->nck, nullptr);
        for (auto &p : a->ck)
            if (e == cudaSuccess) e = cudaMalloc(&p, sbytes);
        a->seg[0].assign(C, nullptr);
        for (auto &p : a->seg[0])
            if (e == cudaSuccess) e = cudaMalloc(&p, sbytes);
        a->bytes += (a->nck + C) * sbytes;
    }
    for (auto &p : a->phi)
        if (e == cudaSuccess) e = cudaMalloc(&p, pbytes);
    a->nslot_init = (ctx->nodes + 255) / 256 * 8;
    if (e == cudaSuccess) e = cudaMalloc(&a->th0, sizeof(double) * ctx->nodes);
    if (e == cudaSuccess) e = cudaMalloc(&a->grad, sizeof(double) * ctx->d * ctx->nodes);
    if (e == cudaSuccess) e = cudaMalloc(&a->h, sizeof(double) * ctx->d * ctx->nodes);
    if (e == cudaSuccess) e = cudaMalloc(&a->slot_step, sizeof(double) * a->ag.nseg);
    if (e == cudaSuccess) e = cudaMalloc(&a->slot_init, sizeof(double) * a->nslot_init);
    if (e == cudaSuccess) e = cudaMalloc(&a->dsum, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&a->dflag, sizeof(int));
    a->bytes += 2 * pbytes + sizeof(double) * ctx->nodes * (1 + 2 * ctx->d);
    if (e != cudaSuccess) {
        free_adj(a);
        return e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;
    }
    if (a->want_nu && a->nck >= 2) {
        // optional: the buffer the next segment is recomputed into while the
        // current one is reversed; without room for it segments are recomputed
        // one at a time, the same launches in the same order within each
        std::vector<void *> s2(C, nullptr);
        for (auto &p : s2)
            if (e == cudaSuccess) e = cudaMalloc(&p, sbytes);
        if (e == cudaSuccess) {
            a->seg[1] = std::move(s2);
            a->nseg_buf = 2;
            a->bytes += C * sbytes;
        } else {
            for (void *p : s2) cudaFree(p);
            if (e != cudaErrorMemoryAllocation) {
                free_adj(a);
                return LB_ECUDA;
            }
            cudaGetLastError();  // an allocation failure leaves no sticky error
        }
    }
    *out = a;
    return LB_OK;
}

lb_status lb_adjoint_destroy(lb_adj *a)
{
    if (!a) return LB_OK;
    cudaStreamSynchronize(a->ctx->stream);
    free_adj(a);
    return LB_OK;
}

lb_status lb_adjoint_forward(lb_adj *a, const double *theta0, double *theta, double *u)
{
    lbk::NvtxRange nvtx_range("lb_adjoint_forward");
    if (!a || !theta0) return LB_EINVAL;
    lb_ctx *c = a->ctx;
    a->ag.mirror = c->geom.mirror;  // the walls may have been set after the workspace was made
    a->forward_done = a->seeded = false;
    a->seg_loaded[0] = a->seg_loaded[1] = -1;
    lb_status st = lb_set_theta0(c, theta0, nullptr);  // FD4 gradient: a function of theta0 alone
    if (st != LB_OK) return st;
    make_adjk(a);  // after lb_set_theta0: the FX64 scale is known now
    a->fwd_gen = c->gen;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(a->th0, theta0, sizeof(double) * c->nodes, cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(a->grad, c->gradtmp, sizeof(double) * c->d * c->nodes, cudaMemcpyDeviceToDevice,
                             c->stream)) != cudaSuccess)
        return acuda(a, e, "lb_adjoint_forward");
    const bool cap = stream_capturing(c->stream);
    for (int64_t k = 0; k * a->C < a->T; ++k) {
        if (a->want_nu &&
            (e = cudaMemcpyAsync(a->ck[k], c->f[c->cur], a->state_bytes, cudaMemcpyDeviceToDevice, c->stream)) !=
                cudaSuccess)
            return acuda(a, e, "lb_adjoint_forward: checkpoint");
        const int64_t n = std::min<int64_t>(a->C, a->T - k * a->C);
        if (n < a->C || cap) {  // a short last segment, or inside the caller's capture: plain launches
            if ((st = lb_step(c, n)) != LB_OK) return st;
            continue;
        }
        const int p = c->cur;
        if (!a->fgraph[p] || a->fgen[p] != c->gen) {
            e = record_graph(c, &a->fgraph[p], [&]() {
                cudaError_t r = cudaSuccess;
                for (int64_t m = 0, q = p; m < n && r == cudaSuccess; ++m, q ^= 1)
                    r = lbk::launch_sweep(c, c->f[q], c->f[q ^ 1]);
                return r;
            });
            if (e != cudaSuccess) return acuda(a, e, "lb_adjoint_forward: record");
            a->fgen[p] = c->gen;
        }
        if ((e = cudaGraphLaunch(a->fgraph[p], c->stream)) != cudaSuccess)
            return acuda(a, e, "lb_adjoint_forward: graph");
        c->cur ^= (int)(n & 1);
        c->step += n;
    }
    if ((theta || u) && (st = lb_macros(c, theta, nullptr, u)) != LB_OK) return st;
    a->forward_done = true;
    return LB_OK;
}

lb_status lb_adjoint_seed(lb_adj *a, const double *dLdu, const double *dLdth)
{
    lbk::NvtxRange nvtx_range("lb_adjoint_seed");
    if (!a) return LB_EINVAL;
    if (!dLdu && !dLdth) return afail(a, LB_EINVAL, "lb_adjoint_seed: dL_du and dL_dtheta are both NULL");
    if (!a->forward_done || a->ctx->step != a->T)
        return afail(a, LB_ESTATE, "lb_adjoint_seed: run lb_adjoint_forward first (and do not step the context)");
    lb_ctx *c = a->ctx;
    cudaError_t e;
    if ((e = cudaMemsetAsync(a->slot_step, 0, sizeof(double) * a->ag.nseg, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(a->slot_init, 0, sizeof(double) * a->nslot_init, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(a->dflag, 0, sizeof(int), c->stream)) != cudaSuccess)
        return acuda(a, e, "lb_adjoint_seed");
    a->pcur = 0;
    if ((e = do_seed(a, dLdu, dLdth)) != cudaSuccess) return acuda(a, e, "lb_adjoint_seed: launch");
    a->done = 0;
    a->seeded = true;
    return LB_OK;
}

lb_status lb_adjoint_step(lb_adj *a, int64_t nsteps)
{
    lbk::NvtxRange nvtx_range("lb_adjoint_step");
    if (!a || nsteps < 0) return LB_EINVAL;
    if (!a->seeded) return afail(a, LB_ESTATE, "lb_adjoint_step: call lb_adjoint_seed first");
    if (a->done + nsteps > a->T) return afail(a, LB_EINVAL, "lb_adjoint_step: more reverse steps than forward");
    if (a->ctx->geom.mirror != a->ag.mirror || a->ctx->gen != a->fwd_gen)
        return afail(a, LB_ESTATE, "lb_adjoint_step: the walls or the viscosity changed since lb_adjoint_forward");
    cudaError_t e;
    lb_ctx *c = a->ctx;
    const bool cap = stream_capturing(c->stream);
    const int64_t C = a->C;
    for (int64_t s = 0; s < nsteps;) {
        const int64_t n = a->T - 1 - a->done;  // producing phi_n from phi_{n+1}
        const int64_t k = n / C;
        if (a->want_nu && !cap && n == k * C + C - 1 && nsteps - s >= C) {
            // a whole segment as one recorded graph: its C reverse steps, the same
            // launches in the same order as below, and beside them (two buffers)
            // the recomputation of segment k - 1, which the next segment needs
            const int b = seg_buf(a, k);
            if (a->seg_loaded[b] != k && (e = load_segment(a, k)) != cudaSuccess)
                return acuda(a, e, "lb_adjoint_step: recompute");
            const int pre = (a->nseg_buf == 2 && k >= 1) ? 1 : 0;
            if (pre && (e = cudaMemcpyAsync(a->seg[b ^ 1][0], a->ck[k - 1], a->state_bytes,
                                            cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
                return acuda(a, e, "lb_adjoint_step: checkpoint");
            const int p = a->pcur;
            cudaGraphExec_t &g = a->rgraph[p][b][pre];
            if (!g || a->rmirror[p][b][pre] != a->ag.mirror || memcmp(&a->rK[p][b][pre], &a->K, sizeof(a->K)) != 0) {
                cudaStream_t s2 = nullptr;
                cudaEvent_t fork = nullptr, join = nullptr;
                e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
                if (e == cudaSuccess)
                    e = record_graph(c, &g, [&]() {
                        cudaError_t r = cudaSuccess;
                        cudaStream_t main = c->stream;
                        if (pre) {  // second branch: the C - 1 sweeps of segment k - 1
                            if ((r = cudaEventRecord(fork, main)) != cudaSuccess ||
                                (r = cudaStreamWaitEvent(s2, fork, 0)) != cudaSuccess)
                                return r;
                            c->stream = s2;
                            for (int64_t m = 1; m < C && r == cudaSuccess; ++m)
                                r = lbk::launch_sweep(c, a->seg[b ^ 1][m - 1], a->seg[b ^ 1][m]);
                            c->stream = main;
                            if (r == cudaSuccess) r = cudaEventRecord(join, s2);
                        }
                        for (int64_t j = C - 1; j >= 0 && r == cudaSuccess; --j) {
                            r = do_step(a, a->seg[b][j]);
                            a->pcur ^= 1;
                        }
                        a->pcur = p;
                        if (pre && r == cudaSuccess) r = cudaStreamWaitEvent(main, join, 0);
                        return r;
                    });
                if (join) cudaEventDestroy(join);
                if (fork) cudaEventDestroy(fork);
                if (s2) cudaStreamDestroy(s2);
                if (e != cudaSuccess) return acuda(a, e, "lb_adjoint_step: record");
                a->rK[p][b][pre] = a->K;
                a->rmirror[p][b][pre] = a->ag.mirror;
            }
            if ((e = cudaGraphLaunch(g, c->stream)) != cudaSuccess) return acuda(a, e, "lb_adjoint_step: graph");
            if (pre) a->seg_loaded[b ^ 1] = k - 1;
            a->pcur ^= (int)(C & 1);
            a->done += C;
            s += C;
            continue;
        }
        const void *Pn = nullptr;
        if (a->want_nu && (e = state_at(a, n, &Pn)) != cudaSuccess) return acuda(a, e, "lb_adjoint_step: recompute");
        if ((e = do_step(a, Pn)) != cudaSuccess) return acuda(a, e, "lb_adjoint_step: launch");
        a->pcur ^= 1;
        ++a->done;
        ++s;
    }
    return LB_OK;
}

lb_status lb_adjoint_result(lb_adj *a, double *dL_dtheta0, double *dL_dnu)
{
    lbk::NvtxRange nvtx_range("lb_adjoint_result");
    if (!a || !dL_dtheta0) return LB_EINVAL;
    if (!a->seeded || a->done != a->T) return afail(a, LB_ESTATE, "lb_adjoint_result: reverse pass incomplete");
    lb_ctx *c = a->ctx;
    cudaError_t e = do_init(a, dL_dtheta0);
    if (e != cudaSuccess) return acuda(a, e, "lb_adjoint_result: init adjoint");
    if (a->fx) {
        int flag = 0;
        if ((e = cudaMemcpyAsync(&flag, a->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
            return acuda(a, e, "lb_adjoint_result");
        if (flag)
            return afail(a, LB_EINVAL, "lb_adjoint_result: the fixed-point adjoint field left its range");
    }
    if (dL_dnu) {
        if (!a->want_nu) return afail(a, LB_EINVAL, "lb_adjoint_result: dL/dnu was not requested");
        lbk::sum_slots_kernel<<<1, 256, 0, c->stream>>>(a->slot_step, a->ag.nseg, a->slot_init, a->nslot_init,
                                                        a->dsum);
        double deps = 0.0;
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(&deps, a->dsum, sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return acuda(a, e, "lb_adjoint_result: eps sum");
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return acuda(a, e, "lb_adjoint_result");
        *dL_dnu = deps * c->dt / (c->dx * c->dx);  // d eps / d nu
        return LB_OK;
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return acuda(a, e, "lb_adjoint_result");
    return LB_OK;
}

lb_status lb_selftest_int_to_f64(const long long *hi, const unsigned long long *lo, int64_t n, double *out128,
                                 double *out64, void *stream)
{
    if (n < 0 || (n > 0 && (!hi || !lo || !out128 || !out64))) return LB_EINVAL;
    if (n == 0) return LB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    lbk::int_to_f64_selftest_kernel<<<nb, 256, 0, st>>>(hi, lo, n, out128, out64);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LB_OK : LB_ECUDA;
}

lb_status lb_adjoint_info(const lb_adj *a, double *info)
{
    if (!a || !info) return LB_EINVAL;
    info[0] = (double)a->T;
    info[1] = (double)a->C;
    info[2] = (double)a->nck;
    info[3] = (double)a->done;
    info[4] = (double)a->bytes;
    return LB_OK;
}

}  // extern "C"
