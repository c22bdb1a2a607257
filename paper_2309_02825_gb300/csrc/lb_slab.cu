// One slab of a grid cut along its slowest axis (include/lb_slab.h): an
// ordinary context over the slab's layers plus one ghost layer on each side,
// and the packing of the populations that cross the cuts.  The sweep, the
// recovery and the sums are the single-grid kernels (the recovery and the
// sum restricted to the owned rows); packing and unpacking are device copies
// of whole layers, one per crossing population.
#include <math.h>

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

// Copy the listed populations' layer `layer` of the current state to (pack)
// or from (unpack) consecutive slots of a buffer.
static cudaError_t copy_layers(lb_slab *s, const std::vector<int> &pops, int64_t layer, void *buf, bool pack)
{
    lb_ctx *c = s->ctx;
    const size_t bytes = (size_t)s->layer_elems * c->elem;
    char *state = (char *)c->f[c->cur];
    for (size_t k = 0; k < pops.size(); ++k) {
        char *st = state + ((size_t)pops[k] * c->geom.slab + (size_t)layer * s->layer_elems) * c->elem;
        char *b = (char *)buf + k * bytes;
        cudaError_t e = pack ? cudaMemcpyAsync(b, st, bytes, cudaMemcpyDeviceToDevice, c->stream)
                             : cudaMemcpyAsync(st, b, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

lb_status lb_slab_pack(lb_slab *s, void *send_down, void *send_up)
{
    lbk::NvtxRange nvtx_range("lb_slab_pack");
    if (!s || !send_down || !send_up) return LB_EINVAL;
    if (!s->ctx->initialized) return sfail(s, LB_ESTATE, "lb_slab_pack: no state (lb_slab_set_theta0 first)");
    cudaError_t e = copy_layers(s, s->up, s->nz, send_up, true);  // last owned layer, moving up
    if (e == cudaSuccess) e = copy_layers(s, s->down, 1, send_down, true);  // first owned layer, moving down
    if (e != cudaSuccess) return scuda(s, e, "lb_slab_pack");
    return LB_OK;
}

lb_status lb_slab_unpack(lb_slab *s, const void *recv_down, const void *recv_up)
{
    lbk::NvtxRange nvtx_range("lb_slab_unpack");
    if (!s || !recv_down || !recv_up) return LB_EINVAL;
    if (!s->ctx->initialized) return sfail(s, LB_ESTATE, "lb_slab_unpack: no state (lb_slab_set_theta0 first)");
    cudaError_t e = copy_layers(s, s->up, 0, const_cast<void *>(recv_down), false);  // from below: lower ghost
    if (e == cudaSuccess) e = copy_layers(s, s->down, s->nz + 1, const_cast<void *>(recv_up), false);
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
