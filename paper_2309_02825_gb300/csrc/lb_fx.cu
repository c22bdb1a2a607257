// 64-bit fixed-point MRT-LB sweep launch and constants (precision LB_FX64);
// the fixed-point collisions themselves are in lb_device.cuh, shared with the
// batched sweep.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so an FP64 collision is
// bound by the FP64 pipe long before HBM.  The update of Eq.
// (distribution-f) is linear with fixed coefficients, so it can run on the
// integer pipes instead: every distribution is stored as round(f * 2^F) in
// an int64, the moment sums theta, J_a, P_aa, P_ab are exact integer
// additions, each of the few products with a relaxation constant (held
// with 64 fractional bits) is rounded to nearest once, and the rest
// population is theta minus all others, which conserves sum theta exactly.
// Recovery (lb_recover.cu) sums the exact integer moments and converts them
// to FP64 once, so J = sum e f carries no cancellation error.
#include <algorithm>

#include "lb_device.cuh"

namespace lbk {

static long long to_fx_coef(double v) { return llrint(ldexp(v, kFxCollBits)); }

CollFx make_coll_fx(const lb_ctx *c)
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

bool fx_constants_ok(const lb_ctx &c)
{
    const double d = c.d;
    const double s2x = c.s2x, s22 = (c.d > 1) ? c.s22 : 1.0, wd = (c.d > 1) ? c.wd : 0.0;
    const double v[5] = {(1.0 - c.s1) / 2.0, (1.0 - s2x) / 2.0, (1.0 - s22) / 4.0,
                         s2x * c.sigma / 2.0 - 2.0 * (d - 1.0) * wd, wd};
    for (double x : v)
        if (!(fabs(x) < 0.5 - 0x1p-30)) return false;
    return true;
}

// The constants with the context's range flag, for the single-grid sweeps.
static CollFxR make_coll_fxr(lb_ctx *c)
{
    CollFxR k;
    static_cast<CollFx &>(k) = make_coll_fx(c);
    k.range = c->dflag + kFlagRange;
    return k;
}

template <class L> static cudaError_t sweep_fx_t(lb_ctx *c, const void *src, void *dst)
{
    constexpr int TH = sweep_threads<long long>();
    const bool flat = sweep_flat(c->geom, L::D, 8);
    const unsigned nb = (unsigned)(((flat ? c->geom.fseg : c->geom.nseg) + TH / 32 - 1) / (TH / 32));
    if constexpr (L::D == 4) {
        if (flat) {
            sweep_flat_kernel<L, long long, CollFxR><<<nb, TH, 0, c->stream>>>(
                (const long long *)src, (long long *)dst, c->geom, make_coll_fxr(c));
            return cudaGetLastError();
        }
    }
    if (c->geom.mirror)
        sweep_kernel<L, long long, CollFxR, true><<<nb, TH, 0, c->stream>>>(
            (const long long *)src, (long long *)dst, c->geom, make_coll_fxr(c));
    else
        sweep_kernel<L, long long, CollFxR><<<nb, TH, 0, c->stream>>>(
            (const long long *)src, (long long *)dst, c->geom, make_coll_fxr(c));
    return cudaGetLastError();
}

__global__ void mulfx_selftest_kernel(const long long *a, const long long *k, int64_t n, long long *out_split,
                                      long long *out_wide)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out_split[i] = mulfx_c(a[i], k[i]);
        const __int128 p = (__int128)a[i] * (__int128)k[i];
        out_wide[i] = (long long)((p + ((__int128)1 << 63)) >> 64);
    }
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

extern "C" lb_status lb_selftest_mulfx(const long long *a, const long long *k, int64_t n, long long *out_split,
                                       long long *out_wide, void *stream)
{
    if (n < 0 || (n > 0 && (!a || !k || !out_split || !out_wide))) return LB_EINVAL;
    if (n == 0) return LB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    lbk::mulfx_selftest_kernel<<<nb, 256, 0, st>>>(a, k, n, out_split, out_wide);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LB_OK : LB_ECUDA;
}
