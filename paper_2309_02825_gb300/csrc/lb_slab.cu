// One slab of a grid cut along its slowest axis (include/lb_slab.h): an
// ordinary context over the slab's layers plus one ghost layer on each side,
// and the packing of the populations that cross the cuts.  The sweep, the
// recovery and the sums are the single-grid kernels (the recovery and the
// sum restricted to the owned rows); packing and unpacking move the crossing
// populations' layers of both directions in one launch each.
#include <math.h>

#include <stdint.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/lb_slab.h"
#include "lb_internal.cuh"

struct lb_slab {
    lb_ctx *ctx = nullptr;
    int d = 0, part = 0, nparts = 1;
    int64_t z0 = 0, nz = 0;         // first owned layer (global), owned layers
    int64_t layer_rows = 0;         // rows of one layer (product of the middle axes)
    int64_t layer_elems = 0;        // values of one layer of one population (layer_rows * pitch)
    std::vector<int> up, down;      // populations with +1 / -1 on the slowest axis
    bool halo_fresh = false;        // unpacked since the last sweep
};

namespace {

lb_status sfail(lb_slab *s, lb_status st, const std::string &m)
{
    if (s && s->ctx) s->ctx->err = m;
    return st;
}

lb_status scuda(lb_slab *s, cudaError_t e, const char *where)
{
    return sfail(s, e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

// Velocities of the lattice with component `sign` on axis a, in lattice order.
template <class L> std::vector<int> crossing(int a, int sign)
{
    std::vector<int> v;
    for (int i = 0; i < L::Q; ++i)
        if (L::E[i][a] == sign) v.push_back(i);
    return v;
}

}  // namespace

extern "C" {

lb_status lb_slab_create(int d, const int64_t *N, int part, int nparts, double nu, double dx, double dt,
                         const lb_relax *rs, int precision, void *stream, lb_slab **out)
{
    lbk::NvtxRange nvtx_range("lb_slab_create");
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (d < 2 || d > 4 || !N || nparts < 1 || part < 0 || part >= nparts) return LB_EINVAL;
    for (int a = 0; a < d; ++a)
        if (N[a] < 1) return LB_EINVAL;
    const int64_t Nz = N[d - 1];
    if (Nz < nparts) return LB_EINVAL;  // every part needs a layer
    lb_slab *s = new (std::nothrow) lb_slab();
    if (!s) return LB_ENOMEM;
    s->d = d;
    s->part = part;
    s->nparts = nparts;
    const int64_t base = Nz / nparts, extra = Nz % nparts;
    s->nz = base + (part < extra ? 1 : 0);
    s->z0 = part * base + (part < extra ? part : extra);
    int64_t Nl[4] = {N[0], d > 1 ? N[1] : 1, d > 2 ? N[2] : 1, d > 3 ? N[3] : 1};
    Nl[d - 1] = s->nz + 2;
    lb_status st = lb_create(d, Nl, nu, dx, dt, rs, precision, stream, &s->ctx);
    if (st != LB_OK) {
        delete s;
        return st;
    }
    const lbk::Geom &g = s->ctx->geom;
    s->layer_rows = g.rows / (s->nz + 2);
    s->layer_elems = s->layer_rows * g.pitch;
    switch (d) {
    case 2:
        s->up = crossing<lbk::D2Q9>(1, 1);
        s->down = crossing<lbk::D2Q9>(1, -1);
        break;
    case 3:
        s->up = crossing<lbk::D3Q19>(2, 1);
        s->down = crossing<lbk::D3Q19>(2, -1);
        break;
    default:
        s->up = crossing<lbk::D4Q33>(3, 1);
        s->down = crossing<lbk::D4Q33>(3, -1);
        break;
    }
    *out = s;
    return LB_OK;
}

lb_status lb_slab_destroy(lb_slab *s)
{
    if (!s) return LB_OK;
    lb_destroy(s->ctx);
    delete s;
    return LB_OK;
}

lb_status lb_slab_info(const lb_slab *s, int64_t *info)
{
    if (!s || !info) return LB_EINVAL;
    info[0] = s->z0;
    info[1] = s->nz;
    info[2] = (int64_t)s->up.size() * s->layer_elems;
    info[3] = (int64_t)s->ctx->elem;
    info[4] = (int64_t)s->up.size();
    info[5] = s->layer_rows * s->ctx->geom.N0;
    return LB_OK;
}

lb_ctx *lb_slab_ctx(lb_slab *s) { return s ? s->ctx : nullptr; }

lb_status lb_slab_set_theta0(lb_slab *s, const double *theta0, const double *grad, double max_abs_theta0)
{
    lbk::NvtxRange nvtx_range("lb_slab_set_theta0");
    if (!s) return LB_EINVAL;
    if (!grad) return sfail(s, LB_EINVAL, "lb_slab_set_theta0: grad theta0 is required for a slab");
    lb_ctx *c = s->ctx;
    if (c->precision == LB_FX64) {
        if (!(max_abs_theta0 > 0.0) || !isfinite(max_abs_theta0))
            return sfail(s, LB_EINVAL, "lb_slab_set_theta0: max |theta0| of the grid must be finite and > 0");
        c->fx_max = max_abs_theta0;
    }
    s->halo_fresh = false;
    const lb_status st = lb_set_theta0(c, theta0, grad);
    c->fx_max = 0.0;
    // the initialisation stores every owned node's P values from the layers
    // it was given, ghost layers included: the first sweep needs no exchange
    if (st == LB_OK) s->halo_fresh = true;
    return st;
}

// One direction of an exchange: the listed populations' layer of the state
// and the buffer whose consecutive slots hold them, in 16-byte vectors (a
// layer's rows are padded to 16 bytes, so every layer and slab starts on a
// vector boundary; the buffers are 16-byte aligned by contract).
struct LayerCopy {
    uint4 *buf;
    int64_t layer_off;  // vector offset of the layer within a population's slab
    int npop;
    int pop[8];
};

// Both directions of a pack (state -> buffers) or an unpack (buffers ->
// state) in one launch: thread t moves vector t of the concatenated slots.
__global__ void slab_copy_kernel(uint4 *__restrict__ state, LayerCopy a, LayerCopy b, int64_t layer_vecs,
                                 int64_t slab_vecs, int pack)
{
    const int64_t na = a.npop * layer_vecs, total = na + b.npop * layer_vecs;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const bool first = t < na;
        const LayerCopy &lc = first ? a : b;
        const int64_t u = first ? t : t - na;
        const int k = (int)(u / layer_vecs);
        uint4 *st = state + lc.pop[k] * slab_vecs + lc.layer_off + (u - k * layer_vecs);
        if (pack)
            lc.buf[u] = *st;
        else
            *st = lc.buf[u];
    }
}

static LayerCopy layer_copy(const lb_slab *s, const std::vector<int> &pops, int64_t layer, void *buf)
{
    LayerCopy lc{};
    lc.buf = (uint4 *)buf;
    lc.layer_off = layer * s->layer_elems * (int64_t)s->ctx->elem / 16;
    lc.npop = (int)pops.size();
    for (size_t k = 0; k < pops.size(); ++k) lc.pop[k] = pops[k];
    return lc;
}

// Move the crossing populations of layers `la` (buffer `ba`, populations
// `pa`) and `lb` (buffer `bb`, populations `pb`) to (pack) or from the
// buffers, on the context's stream.
static cudaError_t copy_layers(lb_slab *s, const std::vector<int> &pa, int64_t la, void *ba, const std::vector<int> &pb,
                               int64_t lb, void *bb, bool pack)
{
    lb_ctx *c = s->ctx;
    const int64_t layer_vecs = s->layer_elems * (int64_t)c->elem / 16, slab_vecs = c->geom.slab * (int64_t)c->elem / 16;
    const int64_t total = (int64_t)(pa.size() + pb.size()) * layer_vecs;
    const unsigned nb = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    slab_copy_kernel<<<nb, 256, 0, c->stream>>>((uint4 *)c->f[c->cur], layer_copy(s, pa, la, ba),
                                                layer_copy(s, pb, lb, bb), layer_vecs, slab_vecs, pack ? 1 : 0);
    return cudaGetLastError();
}

lb_status lb_slab_pack(lb_slab *s, void *send_down, void *send_up)
{
    lbk::NvtxRange nvtx_range("lb_slab_pack");
    if (!s || !send_down || !send_up) return LB_EINVAL;
    if ((((uintptr_t)send_down) | ((uintptr_t)send_up)) & 15u)
        return sfail(s, LB_EINVAL, "lb_slab_pack: buffers must be 16-byte aligned");
    if (!s->ctx->initialized) return sfail(s, LB_ESTATE, "lb_slab_pack: no state (lb_slab_set_theta0 first)");
    // last owned layer moving up, first owned layer moving down
    cudaError_t e = copy_layers(s, s->up, s->nz, send_up, s->down, 1, send_down, true);
    if (e != cudaSuccess) return scuda(s, e, "lb_slab_pack");
    return LB_OK;
}

lb_status lb_slab_unpack(lb_slab *s, const void *recv_down, const void *recv_up)
{
    lbk::NvtxRange nvtx_range("lb_slab_unpack");
    if (!s || !recv_down || !recv_up) return LB_EINVAL;
    if ((((uintptr_t)recv_down) | ((uintptr_t)recv_up)) & 15u)
        return sfail(s, LB_EINVAL, "lb_slab_unpack: buffers must be 16-byte aligned");
    if (!s->ctx->initialized) return sfail(s, LB_ESTATE, "lb_slab_unpack: no state (lb_slab_set_theta0 first)");
    // from below into the lower ghost layer, from above into the upper one
    cudaError_t e = copy_layers(s, s->up, 0, const_cast<void *>(recv_down), s->down, s->nz + 1,
                                const_cast<void *>(recv_up), false);
    if (e != cudaSuccess) return scuda(s, e, "lb_slab_unpack");
    s->halo_fresh = true;
    return LB_OK;
}

lb_status lb_slab_step(lb_slab *s)
{
    if (!s) return LB_EINVAL;
    if (!s->halo_fresh) return sfail(s, LB_ESTATE, "lb_slab_step: exchange the ghost layers first (pack, send, unpack)");
    const lb_status st = lb_step(s->ctx, 1);
    if (st == LB_OK) s->halo_fresh = false;
    return st;
}

lb_status lb_slab_macros(lb_slab *s, double *theta, double *grad, double *u)
{
    lbk::NvtxRange nvtx_range("lb_slab_macros");
    if (!s) return LB_EINVAL;
    lb_ctx *c = s->ctx;
    if (!c->initialized) return sfail(s, LB_ESTATE, "lb_slab_macros: no state");
    if (!s->halo_fresh) return sfail(s, LB_ESTATE, "lb_slab_macros: exchange the ghost layers first");
    if (!theta && !grad && !u) return LB_OK;
    cudaError_t e = lbk::launch_macros_rows(c, c->f[c->cur], theta, grad, u, c->dflag + lbk::kFlagRecover,
                                            s->layer_rows, s->nz * s->layer_rows);
    if (e != cudaSuccess) return scuda(s, e, "lb_slab_macros");
    return lb_check(c);
}

lb_status lb_slab_sum_theta(lb_slab *s, double *out)
{
    if (!s || !out) return LB_EINVAL;
    lb_ctx *c = s->ctx;
    if (!c->initialized) return sfail(s, LB_ESTATE, "lb_slab_sum_theta: no state");
    cudaError_t e = lbk::launch_sum_state_rows(c, c->f[c->cur], c->dout, s->layer_rows, s->nz * s->layer_rows);
    double v = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, c->dout, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return scuda(s, e, "lb_slab_sum_theta");
    if (c->precision == LB_FP32_SHIFTED) v += c->theta_ref * (double)(s->nz * s->layer_rows * c->geom.N0);
    *out = v;
    return LB_OK;
}

}  // extern "C"
