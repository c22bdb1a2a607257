// lb_reduce_static: the error-norm reduction of lb_reduce without any
// device allocation.
//
// Some callers cannot call cudaMalloc: an application whose framework owns
// all device memory through its own caching allocator (a cudaMalloc behind
// its back can fail or fragment the pool), a service certified to a fixed
// device-memory budget up front, or a code path where the implicit device
// synchronisation of an allocation is not allowed.  They have no context
// (lb_create allocates), so this entry point takes plain device pointers
// and keeps its per-block partial sums in a file-scope __device__ array
// that every GPU loading this library holds until the process exits.
#include <math.h>

#include <mutex>

#include "lb_internal.cuh"

namespace lbk {
cudaError_t launch_norms_into(int d, int64_t nodes, const double *theta, const double *u, const double *ex_theta,
                              const double *ex_u, double *partials, int nblocks, double *raw_out,
                              cudaStream_t stream);
}

namespace {

constexpr int kStaticBlocks = 1024;                       // partial rows
constexpr int64_t kStaticMaxNodes = int64_t(1) << 31;     // same limit as lb_create
constexpr int kMaxDevices = 64;

// kStaticBlocks partial rows plus one row for the folded raw sums:
// (1024 + 1) * 16 doubles = 131,200 bytes per device.
static __device__ __align__(256) double g_norms_scratch[(kStaticBlocks + 1) * lbk::kRedSlots];

std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {nullptr};
int g_blocks[kMaxDevices] = {0};

// Per-device set-up: the host-side name g_norms_scratch is only a stand-in
// for the device array, so its device address is looked up with that device
// current.  The lookup is repeated on every call made outside a stream
// capture (a cheap host call), so an address cached before a
// cudaDeviceReset is never reused; inside a capture, where a first lookup
// could load the module, the cached address of an earlier call is used.
cudaError_t scratch_for_current_device(cudaStream_t stream, double **ptr, int *nblocks)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev] || cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norms_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        int nb = 4 * (sms > 0 ? sms : 148);  // the grid lb_reduce uses
        g_blocks[dev] = nb < kStaticBlocks ? nb : kStaticBlocks;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *ptr = g_scratch_addr[dev];
    *nblocks = g_blocks[dev];
    return cudaSuccess;
}

// Turn the folded raw sums into the lb_reduce output layout.
__global__ void finalize_norms_kernel(const double *__restrict__ raw, int d, double nodes, int have_u,
                                      double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int v = 0; v <= d; ++v) {
        const double se = raw[3 * v], mx = raw[3 * v + 1], sx = raw[3 * v + 2];
        const bool have = (v == 0) || have_u;
        out[3 * v + 0] = have ? sqrt(se / nodes) : (double)NAN;
        out[3 * v + 1] = have ? mx : (double)NAN;
        out[3 * v + 2] = have ? (sx > 0 ? sqrt(se / sx) : (se > 0 ? (double)INFINITY : 0.0)) : (double)NAN;
    }
    out[3 * (d + 1)] = raw[3 * (d + 1)];
}

}  // namespace

extern "C" lb_status lb_reduce_static(int d, int64_t nodes, const double *theta, const double *u,
                                      const double *exact_theta, const double *exact_u, double *out,
                                      void *stream)
{
    // Sizes beyond what the static area serves are rejected up front.
    if (d < 1 || d > 3) return LB_EINVAL;
    if (nodes < 1 || nodes > kStaticMaxNodes) return LB_EINVAL;
    if (!theta || !exact_theta || !out) return LB_EINVAL;
    if ((u == nullptr) != (exact_u == nullptr)) return LB_EINVAL;
    double *scratch = nullptr;
    int nb = 0;
    cudaError_t e = scratch_for_current_device((cudaStream_t)stream, &scratch, &nb);
    if (e != cudaSuccess) return LB_ECUDA;
    // Every block overwrites its whole partial row and the fold overwrites
    // the raw row, so nothing has to be cleared between calls.
    double *raw = scratch + (int64_t)kStaticBlocks * lbk::kRedSlots;
    cudaStream_t s = (cudaStream_t)stream;
    e = lbk::launch_norms_into(d, nodes, theta, u, exact_theta, exact_u, scratch, nb, raw, s);
    if (e != cudaSuccess) return LB_ECUDA;
    finalize_norms_kernel<<<1, 32, 0, s>>>(raw, d, (double)nodes, u != nullptr, out);
    if (cudaGetLastError() != cudaSuccess) return LB_ECUDA;
    return LB_OK;
}
