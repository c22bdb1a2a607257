// 64-bit fixed-point MRT-LB sweep and recovery (precision LB_FX64).
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so an FP64 collision is
// bound by the FP64 pipe long before HBM.  The update of Eq.
// (distribution-f) is linear with fixed coefficients, so it can run on the
// integer pipes instead: every distribution is stored as round(f * 2^F) in
// an int64, the moment sums theta, J_a, P_aa, P_ab are exact integer
// additions, each of the few products with a relaxation constant (held
// with 62 fractional bits) is rounded to nearest once, and the rest
// population is theta minus all others, which conserves sum theta exactly.
// Recovery (lb_recover.cu) sums the exact integer moments and converts them
// to FP64 once, so J = sum e f carries no cancellation error.
#include "lb_device.cuh"

namespace lbk {

__device__ __forceinline__ void collide(D1Q3, long long *f, const CollFx &k)
{
    const long long P = f[1] + f[2];
    const long long th = f[0] + P;
    const long long J = f[1] - f[2];
    const long long A = mulfx(P, k.k2) + mulfx(th, k.cA);
    const long long B = mulfx(J, k.k1);
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
    const long long cth = mulfx(th, k.cA);
    const long long Ax = mulfx(Pxx, k.k2) + cth, Bx = mulfx(Jx, k.k1);
    const long long Ay = mulfx(Pyy, k.k2) + cth, By = mulfx(Jy, k.k1);
    const long long wth = mulfx(th, k.wd);
    const long long B3 = mulfx(Pxy, k.k3);
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
    const long long cth = mulfx(th, k.cA);
    const long long wth = mulfx(th, k.wd);
    long long axis = 0, diag = 0;
    {
        const long long A = mulfx(Pxx, k.k2) + cth, B = mulfx(Jx, k.k1);
        f[1] = A + B;
        f[4] = A - B;
        axis += A;
    }
    {
        const long long A = mulfx(Pyy, k.k2) + cth, B = mulfx(Jy, k.k1);
        f[2] = A + B;
        f[5] = A - B;
        axis += A;
    }
    {
        const long long A = mulfx(Pzz, k.k2) + cth, B = mulfx(Jz, k.k1);
        f[3] = A + B;
        f[6] = A - B;
        axis += A;
    }
    {
        const long long B = mulfx(xy.P, k.k3), dp = wth + B, dm = wth - B;
        f[7] = dp; f[9] = dp; f[8] = dm; f[10] = dm;
        diag += dp + dm;
    }
    {
        const long long B = mulfx(xz.P, k.k3), dp = wth + B, dm = wth - B;
        f[11] = dp; f[13] = dp; f[12] = dm; f[14] = dm;
        diag += dp + dm;
    }
    {
        const long long B = mulfx(yz.P, k.k3), dp = wth + B, dm = wth - B;
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
    const long long cth = mulfx(th, k.cA), wth = mulfx(th, k.wd);
    long long rest = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const long long A = mulfx(P[a], k.k2) + cth, Bq = mulfx(J[a], k.k1);
        f[1 + a] = A + Bq;
        f[1 + D + a] = A - Bq;
        rest += A;
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const long long Bq = mulfx(pl[p].P, k.k3), dp = wth + Bq, dm = wth - Bq;
        f[B0 + 4 * p] = dp;
        f[B0 + 4 * p + 1] = dm;
        f[B0 + 4 * p + 2] = dp;
        f[B0 + 4 * p + 3] = dm;
        rest += dp + dm;
    }
    f[0] = th - 2 * rest;
}

static long long to_fx_coef(double v) { return llrint(ldexp(v, kFxCoefBits)); }

static CollFx make_coll_fx(const lb_ctx *c)
{
    const double d = c->d;
    const double s2x = c->s2x, s22 = (c->d > 1) ? c->s22 : 1.0, wd = (c->d > 1) ? c->wd : 0.0;
    CollFx k;
    k.k1 = to_fx_coef((1.0 - c->s1) / 2.0);
    k.k2 = to_fx_coef((1.0 - s2x) / 2.0);
    k.k3 = to_fx_coef((1.0 - s22) / 4.0);
    k.cA = to_fx_coef(s2x * c->sigma / 2.0 - 2.0 * (d - 1.0) * wd);
    k.wd = to_fx_coef(wd);
    return k;
}

template <class L> static cudaError_t sweep_fx_t(lb_ctx *c, const void *src, void *dst)
{
    constexpr int TH = sweep_threads<long long>();
    const unsigned nb = (unsigned)((c->geom.nseg + TH / 32 - 1) / (TH / 32));
    if (c->geom.mirror)
        sweep_kernel<L, long long, CollFx, true><<<nb, TH, 0, c->stream>>>(
            (const long long *)src, (long long *)dst, c->geom, make_coll_fx(c));
    else
        sweep_kernel<L, long long, CollFx><<<nb, TH, 0, c->stream>>>(
            (const long long *)src, (long long *)dst, c->geom, make_coll_fx(c));
    return cudaGetLastError();
}

cudaError_t launch_sweep_fx(lb_ctx *c, const void *src, void *dst)
{
    switch (c->d) {
    case 1: return sweep_fx_t<D1Q3>(c, src, dst);
    case 2: return sweep_fx_t<D2Q9>(c, src, dst);
    case 3: return sweep_fx_t<D3Q19>(c, src, dst);
    default: return sweep_fx_t<D4Q33>(c, src, dst);
    }
}

}  // namespace lbk
