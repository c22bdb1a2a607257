// Batched 2D MRT-LB (include/lb_batch.h): many independent D2Q9 instances.
//
// State: two big buffers; instance j owns q slabs of its own padded layout
// at element offset off_j in both.  A step kernel launch covers one group
// of instances; every block belongs to exactly one instance (its warps take
// consecutive row segments of that instance), so a block reads the
// instance descriptor once and then runs the same pull + collide as the
// single-grid sweep.  Groups are sized so that their two buffers stay in
// L2 while the group runs all its steps back to back; the launches are
// replayed from CUDA graphs.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/lb_batch.h"
#include "lb_device.cuh"

namespace lbk {

// Collision constants of a storage type: floating point, or 64-bit fixed point.
template <typename T> struct CollOf {
    using type = Coll<T>;
};
template <> struct CollOf<long long> {
    using type = CollFx;
};

template <typename T> struct InstDesc {
    Geom g;
    typename CollOf<T>::type k;
    int64_t off;  // element offset of the instance's state in each buffer
};

constexpr int kBatchMaxThreads = 512;

template <class L, typename T>
__global__ void __launch_bounds__(kBatchMaxThreads) batch_sweep_kernel(const InstDesc<T> *__restrict__ inst,
                                                                       const int *__restrict__ blk_inst,
                                                                       const int *__restrict__ blk_seg0,
                                                                       const T *__restrict__ src,
                                                                       T *__restrict__ dst)
{
    constexpr int V = Vec<T>::V;
    const InstDesc<T> D = inst[blk_inst[blockIdx.x]];
    const int lane = threadIdx.x & 31;
    const int64_t seg = (int64_t)blk_seg0[blockIdx.x] + (threadIdx.x >> 5);
    if (seg >= D.g.nseg) return;  // warp-uniform
    const int64_t row = seg / D.g.seg_per_row;
    const int x0 = (int)(seg - row * D.g.seg_per_row) * (32 * V);
    const T *s = src + D.off;
    T *d = dst + D.off;

    T f[L::Q][V];
    gather<L, T>(s, D.g, row, x0, lane, f);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T n[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) n[i] = f[i][v];
        collide(L{}, n, D.k);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) f[i][v] = n[i];
    }
    if (x0 + V * lane >= D.g.pitch) return;  // beyond the row: loads only
    T *dp = d + row * D.g.pitch + x0 + V * lane;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) st_vec(dp + (int64_t)i * D.g.slab, f[i]);
}

// ---------------------------------------------------------------------------
// Temporally blocked sweep: K steps per launch with the state in shared
// memory.  One block owns one tile (tx x ty nodes) of one instance.  It
// loads the tile plus a K-node halo on every side (periodic wrap at the
// instance's edges; a tile wider than its instance wraps onto itself) into
// shared memory, runs K steps there and stores the tile.  Blocks only read
// the source buffer and write disjoint tiles of the destination buffer, and
// the launch boundary orders launches: there is no wait between blocks.
//
// One shared buffer serves all K steps (the "AA" access pattern): a pull
// step reads node x's pre-collision values from the neighbours, f_i(x) in
// slot opp(i) of x - e_i, and writes f*_i(x) into slot i of x + e_i; a local
// step reads f_i(x) from x's own slot i and writes f*_i(x) into its own slot
// opp(i).  In either step the slots a node reads are exactly the slots it
// writes, and no two nodes share a slot, so the update is in place without
// races; steps alternate pull, local, pull, ...  The stored P form, f*_i(y)
// held as P_i(y), is loaded into slot opp(i) of y, which is the state a pull
// step expects; after an even number of steps it is in that form again,
// after an odd number P_i(y) sits in slot i of y + e_i.  Step s updates the
// nodes s or more away from the loaded region's border: their K-step
// dependency cone (one node per step) lies inside it, and after K steps the
// tile itself is valid; nodes nearer the border only ever hand garbage to
// nodes that are not valid either.
// HBM traffic per lattice update falls from 2 q sizeof(T) to
// q sizeof(T) [(tx + 2K)(ty + 2K) + tx ty] / (K tx ty); the halo nodes'
// recomputation is the price.  The arithmetic per node is the single-grid
// collision on the same inputs, so results are bit-identical to it.
// ---------------------------------------------------------------------------
struct TileDesc {
    int inst;      // instance
    int x0, y0;    // tile origin (nodes)
    int tx, ty;    // tile size (nodes)
};

// Asynchronous global -> shared copy of one value at a 32-bit shared address.
template <typename T> __device__ __forceinline__ void cp_async_elem(unsigned dst, const T *src)
{
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

// Shared-memory loads and stores at a 32-bit shared address plus a
// compile-time byte offset.
template <typename T, int OFF> __device__ __forceinline__ T lds(unsigned a)
{
    T v;
    if constexpr (std::is_same<T, float>::value)
        asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF) : "memory");
    else if constexpr (std::is_same<T, double>::value)
        asm volatile("ld.shared.f64 %0, [%1+%2];" : "=d"(v) : "r"(a), "n"(OFF) : "memory");
    else
        asm volatile("ld.shared.s64 %0, [%1+%2];" : "=l"(v) : "r"(a), "n"(OFF) : "memory");
    return v;
}
template <int OFF> __device__ __forceinline__ void sts(unsigned a, float v)
{
    asm volatile("st.shared.f32 [%0+%1], %2;" ::"r"(a), "n"(OFF), "f"(v) : "memory");
}
template <int OFF> __device__ __forceinline__ void sts(unsigned a, double v)
{
    asm volatile("st.shared.f64 [%0+%1], %2;" ::"r"(a), "n"(OFF), "d"(v) : "memory");
}
template <int OFF> __device__ __forceinline__ void sts(unsigned a, long long v)
{
    asm volatile("st.shared.s64 [%0+%1], %2;" ::"r"(a), "n"(OFF), "l"(v) : "memory");
}

__device__ __forceinline__ int wrap_index(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Shared-memory layout of a blocked tile: W = tx + 2K by H = ty + 2K nodes,
// row-major, each node's Q values contiguous (Q sizeof(T) bytes: an odd
// number of 4-byte words for D2Q9, so a warp's 32 consecutive nodes hit 32
// different banks).  Every slot of a node and of its row neighbours is then
// a compile-time offset from one of three row bases.
__host__ __device__ inline size_t tb_smem_bytes(int q, int elem, int W, int H)
{
    return (size_t)q * W * H * elem;
}

template <class L, typename T, int TH>
__global__ void __launch_bounds__(TH, TH <= 512 ? 2 : 1) batch_tb_kernel(const InstDesc<T> *__restrict__ inst,
                                                                     const TileDesc *__restrict__ tiles,
                                                                     const T *__restrict__ src, T *__restrict__ dst,
                                                                     int K, int *__restrict__ range)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int Q = L::Q, NW = TH / 32;
    constexpr int E = (int)sizeof(T), NB = Q * E;  // bytes per value, per node
    const TileDesc t = tiles[blockIdx.x];
    const InstDesc<T> D = inst[t.inst];
    const int W = t.tx + 2 * K, H = t.ty + 2 * K;
    const int gx0 = t.x0 - K;  // global column of tile column 0 (may be < 0)
    const unsigned smA = (unsigned)__cvta_generic_to_shared(smem_raw);
    const unsigned rowB = (unsigned)(W * NB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // Load the tile and its halo, P_i(y) into slot opp(i) of y (periodic wrap).
    const T *s = src + D.off;
    const bool inner = gx0 >= 0 && gx0 + W <= D.g.N0;  // no column of this tile wraps
    for (int r = warp; r < H; r += NW) {
        const T *grow = s + (int64_t)wrap_index(t.y0 - K + r, D.g.N1) * D.g.pitch;
        const unsigned srow = smA + (unsigned)r * rowB;
        for (int c = lane; c < W; c += 32) {
            int gx = gx0 + c;
            if (!inner) gx = wrap_index(gx, D.g.N0);
            const unsigned a = srow + (unsigned)(c * NB);
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                cp_async_elem(a + (unsigned)(reflect_pop<L>(i, 3) * E), grow + (int64_t)i * D.g.slab + gx);
            });
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    // K steps in place, alternating pull and local.
    for (int st = 0; st < K; ++st) {
        // this thread's nodes of the RW x RH region: flat indices tid, tid + TH,
        // ... walked as (row, column) without a division per node
        const int m = st + 1, RW = W - 2 * m, RH = H - 2 * m;
        const int dr = TH / RW, dc = TH - dr * RW;
        int r = (int)threadIdx.x / RW, c = (int)threadIdx.x - r * RW;
        if ((st & 1) == 0) {  // pull: load from slot opp(i) of x - e_i, store to slot i of x + e_i
            for (; r < RH; r += dr, c += dc) {
                if (c >= RW) {
                    c -= RW;
                    ++r;
                    if (r >= RH) break;
                }
                const unsigned nb = smA + (unsigned)((r + m) * W + (c + m)) * NB;
                const unsigned rb[3] = {nb - rowB, nb, nb + rowB};  // rows y - 1, y, y + 1
                T f[Q];
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int ex = L::E[i][0], ey = L::E[i][1], o = reflect_pop<L>(i, 3);
                    f[i] = lds<T, (-ex * Q + o) * E>(rb[1 - ey]);
                });
                collide(L{}, f, D.k);
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int ex = L::E[i][0], ey = L::E[i][1];
                    sts<(ex * Q + i) * E>(rb[1 + ey], f[i]);
                });
            }
        } else {  // local: load from slot i of x, store to slot opp(i) of x
            for (; r < RH; r += dr, c += dc) {
                if (c >= RW) {
                    c -= RW;
                    ++r;
                    if (r >= RH) break;
                }
                const unsigned nb = smA + (unsigned)((r + m) * W + (c + m)) * NB;
                T f[Q];
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    f[i] = lds<T, i * E>(nb);
                });
                collide(L{}, f, D.k);
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    sts<reflect_pop<L>(i, 3) * E>(nb, f[i]);
                });
            }
        }
        __syncthreads();
    }

    // Store the tile, P_i(z) for z in the tile: after an even number of steps
    // from slot opp(i) of z, after an odd number from slot i of z + e_i.
    T *d = dst + D.off;
    const bool odd = (K & 1) != 0;
    unsigned acc = 0u;  // fixed point: OR of the high words + 2^29 of the stored values (|v| < 2^61 check)
    for (int r = warp; r < t.ty; r += NW) {
        T *grow = d + (int64_t)(t.y0 + r) * D.g.pitch + t.x0;
        const unsigned rb[3] = {smA + (unsigned)(r + K - 1) * rowB, smA + (unsigned)(r + K) * rowB,
                                smA + (unsigned)(r + K + 1) * rowB};
        for (int c = lane; c < t.tx; c += 32) {
            const unsigned cb = (unsigned)((c + K) * NB);
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int ex = L::E[i][0], ey = L::E[i][1], o = reflect_pop<L>(i, 3);
                const T v = odd ? lds<T, (ex * Q + i) * E>(rb[1 + ey] + cb) : lds<T, o * E>(rb[1] + cb);
                if constexpr (std::is_same<T, long long>::value)
                    acc |= (unsigned)((unsigned long long)v >> 32) + 0x20000000u;
                grow[(int64_t)i * D.g.slab + c] = v;
            });
        }
    }
    if constexpr (std::is_same<T, long long>::value) {
        if (range && __any_sync(0xffffffffu, acc >= 0x40000000u) && lane == 0) atomicOr(range, 1);
    }
}

// Per-instance error sums: one block per instance, FP64, fixed order.
__global__ void __launch_bounds__(kRedThreads) batch_errors_kernel(const int64_t *__restrict__ node_off,
                                                                   const double *__restrict__ th,
                                                                   const double *__restrict__ u,
                                                                   const double *__restrict__ eth,
                                                                   const double *__restrict__ eu,
                                                                   int64_t total_nodes, double *__restrict__ out)
{
    const int j = blockIdx.x;
    const int64_t n0 = node_off[j], n1 = node_off[j + 1];
    double a[4] = {0.0, 0.0, 0.0, 0.0};  // sum e_theta^2, sum |e_u|^2, max|e_theta|, max|e_u|
    for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
        const double et = th[n] - eth[n];
        a[0] += et * et;
        a[2] = fmax(a[2], fabs(et));
        if (u) {
            // components of instance j: x block then y block, each n1 - n0 long
            const int64_t m = n - n0;
            const double ex = u[2 * n0 + m] - eu[2 * n0 + m];
            const double ey = u[2 * n0 + (n1 - n0) + m] - eu[2 * n0 + (n1 - n0) + m];
            a[1] += ex * ex + ey * ey;
            a[3] = fmax(a[3], fmax(fabs(ex), fabs(ey)));
        }
    }
    __shared__ double sh[4][kRedThreads];
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nn = (double)(n1 - n0);
        out[4 * j + 0] = sqrt(sh[0][0] / nn);
        out[4 * j + 1] = sqrt(sh[1][0] / nn);
        out[4 * j + 2] = sh[2][0];
        out[4 * j + 3] = sh[3][0];
    }
    (void)total_nodes;
}

// max |theta0| of each instance (one block per instance): the fixed-point scale.
__global__ void __launch_bounds__(kRedThreads) batch_maxabs_kernel(const int64_t *__restrict__ node_off,
                                                                   const double *__restrict__ th,
                                                                   double *__restrict__ out)
{
    __shared__ double sh[kRedThreads];
    const int j = blockIdx.x;
    double m = 0.0;
    for (int64_t n = node_off[j] + threadIdx.x; n < node_off[j + 1]; n += blockDim.x) m = fmax(m, fabs(th[n]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = sh[0];
}

}  // namespace lbk

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

struct Group {
    std::vector<int> members;
    int64_t bytes = 0;
    int nblocks = 0;
    int *d_blk_inst = nullptr;
    int *d_blk_seg0 = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by starting buffer
};

constexpr int kGraphSteps = 32;  // launches per recorded graph (even)

}  // namespace

struct lb_batch {
    int count = 0;
    int precision = LB_FP32_SHIFTED;
    size_t elem = 4;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<lb_ctx> inst;  // host views: parameters + geometry per instance
    std::vector<int64_t> off, node_off;
    int64_t total_elems = 0, total_nodes = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    void *d_desc = nullptr;
    int64_t *d_node_off = nullptr;
    double *d_err = nullptr;
    int *d_flag = nullptr;
    double *gradtmp = nullptr;
    double budget = 0;
    int threads = 256;
    bool use_graph = true;
    std::vector<Group> groups;
    // temporal blocking (lb_batch_set_blocking): tb_k steps per launch; 0 = one launch per step
    int tb_k = 0, tb_tile = 0, tb_threads = 512;
    int ntiles = 0, tb_maxw = 0, tb_maxh = 0;  // tile count, largest tile (without halo)
    lbk::TileDesc *d_tiles = nullptr;
    cudaGraphExec_t tb_graph[2] = {nullptr, nullptr};  // kTbGraphLaunches blocked launches, by starting buffer
    bool initialized = false;
    std::string err;
};

namespace {

lb_status bfail(lb_batch *b, lb_status s, const std::string &m)
{
    if (b) b->err = m;
    return s;
}

lb_status bcuda(lb_batch *b, cudaError_t e, const char *where)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

void free_groups(lb_batch *b)
{
    for (Group &g : b->groups) {
        cudaFree(g.d_blk_inst);
        cudaFree(g.d_blk_seg0);
        for (auto &ge : g.graph)
            if (ge) cudaGraphExecDestroy(ge);
    }
    b->groups.clear();
}

void free_tiles(lb_batch *b)
{
    cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    for (auto &ge : b->tb_graph)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
    b->ntiles = 0;
    b->tb_k = 0;
}

void free_batch(lb_batch *b)
{
    if (!b) return;
    free_groups(b);
    free_tiles(b);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->d_desc);
    cudaFree(b->d_node_off);
    cudaFree(b->d_err);
    cudaFree(b->d_flag);
    cudaFree(b->gradtmp);
    delete b;
}

template <typename T> cudaError_t upload_desc(lb_batch *b)
{
    std::vector<lbk::InstDesc<T>> h(b->count);
    for (int j = 0; j < b->count; ++j) {
        h[j].g = b->inst[j].geom;
        if constexpr (std::is_same<T, long long>::value)
            h[j].k = lbk::make_coll_fx(&b->inst[j]);
        else
            h[j].k = lbk::make_coll<T>(b->inst[j]);
        h[j].off = b->off[j];
    }
    cudaError_t e = cudaMalloc(&b->d_desc, sizeof(lbk::InstDesc<T>) * b->count);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(b->d_desc, h.data(), sizeof(lbk::InstDesc<T>) * b->count, cudaMemcpyHostToDevice);
}

// Launch one step for group g from buffer `from`.
cudaError_t launch_group(lb_batch *b, const Group &g, int from, cudaStream_t s)
{
    if (g.nblocks == 0) return cudaSuccess;
    if (b->precision == LB_FP64)
        lbk::batch_sweep_kernel<lbk::D2Q9, double><<<g.nblocks, b->threads, 0, s>>>(
            (const lbk::InstDesc<double> *)b->d_desc, g.d_blk_inst, g.d_blk_seg0, (const double *)b->buf[from],
            (double *)b->buf[from ^ 1]);
    else if (b->precision == LB_FX64)
        lbk::batch_sweep_kernel<lbk::D2Q9, long long><<<g.nblocks, b->threads, 0, s>>>(
            (const lbk::InstDesc<long long> *)b->d_desc, g.d_blk_inst, g.d_blk_seg0,
            (const long long *)b->buf[from], (long long *)b->buf[from ^ 1]);
    else
        lbk::batch_sweep_kernel<lbk::D2Q9, float><<<g.nblocks, b->threads, 0, s>>>(
            (const lbk::InstDesc<float> *)b->d_desc, g.d_blk_inst, g.d_blk_seg0, (const float *)b->buf[from],
            (float *)b->buf[from ^ 1]);
    return cudaGetLastError();
}

// Tiles of one N0 x N1 instance: each axis cut into ceil(N / tile)
// near-equal tiles.
void append_tiles(std::vector<lbk::TileDesc> &tv, int inst, int n0, int n1, int tile, int &maxw, int &maxh)
{
    const int ntx = (n0 + tile - 1) / tile, nty = (n1 + tile - 1) / tile;
    const int tx = (n0 + ntx - 1) / ntx, ty = (n1 + nty - 1) / nty;
    maxw = std::max(maxw, tx);
    maxh = std::max(maxh, ty);
    for (int y0 = 0; y0 < n1; y0 += ty)
        for (int x0 = 0; x0 < n0; x0 += tx) tv.push_back({inst, x0, y0, std::min(tx, n0 - x0), std::min(ty, n1 - y0)});
}

constexpr int kTbGraphLaunches = 16;  // blocked launches per recorded graph (even)

template <typename T, int TH> const void *tb_kernel()
{
    return (const void *)lbk::batch_tb_kernel<lbk::D2Q9, T, TH>;
}

template <typename T> const void *tb_kernel_for(int threads)
{
    return threads == 256 ? tb_kernel<T, 256>() : (threads == 512 ? tb_kernel<T, 512>() : tb_kernel<T, 1024>());
}

const void *tb_kernel_prec(int precision, int threads)
{
    if (precision == LB_FP64) return tb_kernel_for<double>(threads);
    if (precision == LB_FX64) return tb_kernel_for<long long>(threads);
    return tb_kernel_for<float>(threads);
}

const void *tb_kernel_of(const lb_batch *b, int threads) { return tb_kernel_prec(b->precision, threads); }

size_t tb_smem(const lb_batch *b, int K)
{
    return lbk::tb_smem_bytes(9, (int)b->elem, b->tb_maxw + 2 * K, b->tb_maxh + 2 * K);
}

// One blocked launch of K steps over every tile, from buffer `from`.
cudaError_t launch_tb(lb_batch *b, int from, int K, cudaStream_t s)
{
    int *range = nullptr;
    void *args[] = {&b->d_desc, &b->d_tiles, &b->buf[from], &b->buf[from ^ 1], &K, &range};
    return cudaLaunchKernel(tb_kernel_of(b, b->tb_threads), dim3((unsigned)b->ntiles), dim3((unsigned)b->tb_threads),
                            args, tb_smem(b, K), s);
}

// Tile every instance for blocked launches of K steps: an axis of N nodes is
// cut into ceil(N / tile) near-equal tiles.  The largest tile plus its halo
// must fit the device's shared memory per block.
lb_status build_tiles(lb_batch *b, int K, int tile, int threads)
{
    cudaError_t e = cudaStreamSynchronize(b->stream);  // tables and graphs may be in use
    if (e != cudaSuccess) return bcuda(b, e, "lb_batch_set_blocking");
    free_tiles(b);
    if (K == 0) return LB_OK;
    std::vector<lbk::TileDesc> tv;
    int maxw = 0, maxh = 0;
    for (int j = 0; j < b->count; ++j) append_tiles(tv, j, (int)b->inst[j].N[0], (int)b->inst[j].N[1], tile, maxw, maxh);
    if (tv.size() > 0x7fffffff) return bfail(b, LB_EINVAL, "lb_batch_set_blocking: too many tiles");
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device)) != cudaSuccess)
        return bcuda(b, e, "lb_batch_set_blocking");
    const size_t need = lbk::tb_smem_bytes(9, (int)b->elem, maxw + 2 * K, maxh + 2 * K);
    if (need > (size_t)optin)
        return bfail(b, LB_EINVAL, "lb_batch_set_blocking: tile plus halo exceeds the shared memory per block");
    if ((e = cudaFuncSetAttribute(tb_kernel_of(b, threads), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)need)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_tiles, sizeof(lbk::TileDesc) * tv.size())) != cudaSuccess ||
        (e = cudaMemcpy(b->d_tiles, tv.data(), sizeof(lbk::TileDesc) * tv.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return bcuda(b, e, "lb_batch_set_blocking: tile table");
    b->ntiles = (int)tv.size();
    b->tb_maxw = maxw;
    b->tb_maxh = maxh;
    b->tb_k = K;
    b->tb_tile = tile;
    b->tb_threads = threads;
    return LB_OK;
}

// Record kTbGraphLaunches blocked launches of tb_k steps starting from buffer `from`.
cudaError_t record_tb_graph(lb_batch *b, int from)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int p = from;
        for (int k = 0; k < kTbGraphLaunches && e == cudaSuccess; ++k) {
            e = launch_tb(b, p, b->tb_k, cs);
            p ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->tb_graph[from], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return e;
}

// Build groups and block tables for (budget, threads).  budget <= 0: every
// instance alone; budget >= total: one group.
lb_status build_schedule(lb_batch *b, double budget, int threads, bool use_graph)
{
    free_groups(b);
    b->budget = budget;
    b->threads = threads;
    b->use_graph = use_graph;
    std::vector<int> order(b->count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return b->inst[a].geom.slab > b->inst[c].geom.slab; });
    // first-fit decreasing on 2 * state bytes
    for (int j : order) {
        const int64_t bytes = 2 * (int64_t)b->inst[j].q * b->inst[j].geom.slab * (int64_t)b->elem;
        bool placed = false;
        if (budget > 0)
            for (Group &g : b->groups)
                if (g.bytes + bytes <= budget) {
                    g.members.push_back(j);
                    g.bytes += bytes;
                    placed = true;
                    break;
                }
        if (!placed) {
            Group g;
            g.members.push_back(j);
            g.bytes = bytes;
            b->groups.push_back(g);
        }
    }
    const int warps = threads / 32;
    for (Group &g : b->groups) {
        std::vector<int> bi, bs;
        for (int j : g.members) {
            const int64_t nseg = b->inst[j].geom.nseg;
            for (int64_t s0 = 0; s0 < nseg; s0 += warps) {
                bi.push_back(j);
                bs.push_back((int)s0);
            }
        }
        g.nblocks = (int)bi.size();
        cudaError_t e;
        if ((e = cudaMalloc(&g.d_blk_inst, sizeof(int) * bi.size())) != cudaSuccess ||
            (e = cudaMalloc(&g.d_blk_seg0, sizeof(int) * bs.size())) != cudaSuccess ||
            (e = cudaMemcpy(g.d_blk_inst, bi.data(), sizeof(int) * bi.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(g.d_blk_seg0, bs.data(), sizeof(int) * bs.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bcuda(b, e, "lb_batch: schedule tables");
    }
    return LB_OK;
}

// Record kGraphSteps launches of group g starting from buffer `from`.
cudaError_t record_graph(lb_batch *b, Group &g, int from)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int p = from;
        for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
            e = launch_group(b, g, p, cs);
            p ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.graph[from], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return e;
}

cudaError_t run_steps(lb_batch *b, int64_t n)
{
    cudaError_t e = cudaSuccess;
    if (b->tb_k > 0) {
        // blocked: launches of tb_k steps (recorded in graphs), then one launch for the remainder
        int64_t launches = n / b->tb_k;
        const int rem = (int)(n % b->tb_k);
        if (b->use_graph) {
            while (launches >= kTbGraphLaunches) {
                if (!b->tb_graph[b->cur] && (e = record_tb_graph(b, b->cur)) != cudaSuccess) return e;
                if ((e = cudaGraphLaunch(b->tb_graph[b->cur], b->stream)) != cudaSuccess) return e;
                launches -= kTbGraphLaunches;  // even: parity unchanged
            }
        }
        for (; launches > 0; --launches) {
            if ((e = launch_tb(b, b->cur, b->tb_k, b->stream)) != cudaSuccess) return e;
            b->cur ^= 1;
        }
        if (rem > 0) {
            if ((e = launch_tb(b, b->cur, rem, b->stream)) != cudaSuccess) return e;
            b->cur ^= 1;
        }
        return cudaSuccess;
    }
    for (Group &g : b->groups) {
        int p = b->cur;
        int64_t left = n;
        if (b->use_graph) {
            while (left >= kGraphSteps) {
                if (!g.graph[p]) {
                    e = record_graph(b, g, p);
                    if (e != cudaSuccess) return e;
                }
                e = cudaGraphLaunch(g.graph[p], b->stream);
                if (e != cudaSuccess) return e;
                left -= kGraphSteps;  // even: parity unchanged
            }
        }
        for (; left > 0; --left) {
            e = launch_group(b, g, p, b->stream);
            if (e != cudaSuccess) return e;
            p ^= 1;
        }
    }
    if (n & 1) b->cur ^= 1;
    return e;
}

}  // namespace

// ---------------------------------------------------------------------------
// Blocked sweeps of a single 2D periodic grid: the batched blocked kernel on
// a batch of one instance (the context's own buffers, offset 0).
// ---------------------------------------------------------------------------
namespace lbk {

template <typename T> static cudaError_t upload_single_desc(lb_ctx *c)
{
    InstDesc<T> h;
    h.g = c->geom;
    if constexpr (std::is_same<T, long long>::value)
        h.k = make_coll_fx(c);
    else
        h.k = make_coll<T>(*c);
    h.off = 0;
    cudaError_t e = cudaSuccess;
    if (!c->tb_desc) e = cudaMalloc(&c->tb_desc, sizeof(InstDesc<long long>) > sizeof(InstDesc<double>)
                                                       ? sizeof(InstDesc<long long>)
                                                       : sizeof(InstDesc<double>));
    if (e == cudaSuccess) e = cudaMemcpy(c->tb_desc, &h, sizeof(h), cudaMemcpyHostToDevice);
    return e;
}

void blocked_release(lb_ctx *c)
{
    for (auto &ge : c->tb_graph)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
    cudaFree(c->tb_tiles);
    cudaFree(c->tb_desc);
    c->tb_tiles = nullptr;
    c->tb_desc = nullptr;
    c->tb_k = c->tb_tile = c->tb_threads = c->tb_ntiles = 0;
}

cudaError_t blocked_setup(lb_ctx *c, int K, int tile, int threads, bool *fits)
{
    *fits = true;
    blocked_release(c);
    if (K == 0) return cudaSuccess;
    std::vector<TileDesc> tv;
    int maxw = 0, maxh = 0;
    append_tiles(tv, 0, (int)c->N[0], (int)c->N[1], tile, maxw, maxh);
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (e != cudaSuccess) return e;
    const size_t need = tb_smem_bytes(9, (int)c->elem, maxw + 2 * K, maxh + 2 * K);
    if (need > (size_t)optin || tv.size() > 0x7fffffff) {
        *fits = false;
        return cudaSuccess;
    }
    if ((e = cudaFuncSetAttribute(tb_kernel_prec(c->precision, threads), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)need)) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&c->tb_tiles, sizeof(TileDesc) * tv.size())) != cudaSuccess ||
        (e = cudaMemcpy(c->tb_tiles, tv.data(), sizeof(TileDesc) * tv.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    e = c->precision == LB_FP64 ? upload_single_desc<double>(c)
                                : (c->precision == LB_FX64 ? upload_single_desc<long long>(c) : upload_single_desc<float>(c));
    if (e != cudaSuccess) return e;
    c->tb_k = K;
    c->tb_tile = tile;
    c->tb_threads = threads;
    c->tb_ntiles = (int)tv.size();
    c->tb_maxw = maxw;
    c->tb_maxh = maxh;
    return cudaSuccess;
}

cudaError_t blocked_launch(lb_ctx *c, const void *src, void *dst, int K, cudaStream_t s)
{
    int *range = c->precision == LB_FX64 ? c->dflag + kFlagRange : nullptr;
    void *args[] = {&c->tb_desc, &c->tb_tiles, (void *)&src, &dst, &K, &range};
    const size_t smem = tb_smem_bytes(9, (int)c->elem, c->tb_maxw + 2 * K, c->tb_maxh + 2 * K);
    return cudaLaunchKernel(tb_kernel_prec(c->precision, c->tb_threads), dim3((unsigned)c->tb_ntiles),
                            dim3((unsigned)c->tb_threads), args, smem, s);
}

}  // namespace lbk

extern "C" {

lb_status lb_batch_create(int count, const int64_t *N, const double *nu, const double *dx, const double *dt,
                          const lb_relax *rs, int precision, void *stream, lb_batch **out)
{
    lbk::NvtxRange nvtx_range("lb_batch_create");
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (count < 1 || count > 65536 || !N || !nu || !dx || !dt) return LB_EINVAL;
    if (precision != LB_FP32_SHIFTED && precision != LB_FP64 && precision != LB_FX64) return LB_EINVAL;
    lb_batch *b = new (std::nothrow) lb_batch();
    if (!b) return LB_ENOMEM;
    b->count = count;
    b->precision = precision;
    b->elem = precision == LB_FP32_SHIFTED ? 4 : 8;
    b->stream = (cudaStream_t)stream;
    cudaGetDevice(&b->device);
    b->inst.resize(count);
    b->off.resize(count);
    b->node_off.resize(count + 1);
    const int V = precision == LB_FP32_SHIFTED ? lbk::Vec<float>::V : lbk::Vec<double>::V;
    int64_t off = 0, noff = 0;
    for (int j = 0; j < count; ++j) {
        lb_ctx &c = b->inst[j];
        const int64_t n0 = N[2 * j], n1 = N[2 * j + 1];
        if (n0 < 1 || n1 < 1 || n0 > 65536 || n1 > 65536 || !(nu[j] > 0) || !(dx[j] > 0) || !(dt[j] > 0) ||
            !isfinite(nu[j]) || !isfinite(dx[j]) || !isfinite(dt[j])) {
            free_batch(b);
            return LB_EINVAL;
        }
        c.d = 2;
        c.q = 9;
        c.N[0] = n0;
        c.N[1] = n1;
        c.N[2] = 1;
        c.N[3] = 1;
        c.nodes = n0 * n1;
        c.precision = precision;
        c.nu = nu[j];
        c.dx = dx[j];
        c.dt = dt[j];
        c.c = dx[j] / dt[j];
        c.eps = nu[j] * dt[j] / (dx[j] * dx[j]);
        if (!lbk::derive_params(c, rs ? &rs[j] : nullptr) || (precision == LB_FX64 && !lbk::fx_constants_ok(c))) {
            free_batch(b);
            return LB_EINVAL;
        }
        c.elem = b->elem;
        c.geom = lbk::make_geom(n0, n1, 1, 1, V);
        const lbk::Geom &g = c.geom;
        c.stream = b->stream;
        c.device = b->device;
        b->off[j] = off;
        b->node_off[j] = noff;
        off += (int64_t)c.q * g.slab;
        noff += c.nodes;
    }
    b->node_off[count] = noff;
    b->total_elems = off;
    b->total_nodes = noff;
    cudaError_t e;
    for (int k = 0; k < 2; ++k) {
        const size_t bytes = b->elem * ((size_t)off + lbk::kSlackElems);
        if ((e = cudaMalloc(&b->buf[k], bytes)) != cudaSuccess ||
            (e = cudaMemsetAsync(b->buf[k], 0, bytes, b->stream)) != cudaSuccess) {
            free_batch(b);
            return e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;
        }
    }
    e = precision == LB_FP64 ? upload_desc<double>(b)
                             : (precision == LB_FX64 ? upload_desc<long long>(b) : upload_desc<float>(b));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_node_off, sizeof(int64_t) * (count + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_node_off, b->node_off.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(double) * 4 * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_flag, sizeof(int) * 2);
    if (e != cudaSuccess) {
        free_batch(b);
        return e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;
    }
    for (int j = 0; j < count; ++j) {
        b->inst[j].f[0] = (char *)b->buf[0] + b->elem * b->off[j];
        b->inst[j].f[1] = (char *)b->buf[1] + b->elem * b->off[j];
    }
    // Default schedule: groups of at most 96 MB (A + B) so each stays in L2.
    lb_status st = build_schedule(b, 96e6, 256, true);
    if (st != LB_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch *b)
{
    if (!b) return LB_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return LB_OK;
}

lb_status lb_batch_set_theta_ref(lb_batch *b, const double *tr)
{
    if (!b || !tr) return LB_EINVAL;
    for (int j = 0; j < b->count; ++j) {
        if (!isfinite(tr[j])) return bfail(b, LB_EINVAL, "lb_batch_set_theta_ref: non-finite value");
        b->inst[j].theta_ref = tr[j];
    }
    return LB_OK;
}

lb_status lb_batch_set_theta0(lb_batch *b, const double *theta0, const double *grad0)
{
    lbk::NvtxRange nvtx_range("lb_batch_set_theta0");
    if (!b) return LB_EINVAL;
    if (!theta0) return bfail(b, LB_EINVAL, "lb_batch_set_theta0: theta0 is NULL");
    b->initialized = false;
    cudaError_t e;
    if (!grad0) {
        if (!b->gradtmp && (e = cudaMalloc(&b->gradtmp, sizeof(double) * 2 * b->total_nodes)) != cudaSuccess)
            return bcuda(b, e, "lb_batch_set_theta0: gradient buffer");
    }
    if ((e = cudaMemsetAsync(b->d_flag, 0, sizeof(int) * 2, b->stream)) != cudaSuccess)
        return bcuda(b, e, "lb_batch_set_theta0");
    if (b->precision == LB_FX64) {
        // each instance's scale as for one grid: max|theta0_j| 2^F_j < 2^59
        std::vector<double> mx(b->count);
        lbk::batch_maxabs_kernel<<<b->count, lbk::kRedThreads, 0, b->stream>>>(b->d_node_off, theta0, b->d_err);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(mx.data(), b->d_err, sizeof(double) * b->count, cudaMemcpyDeviceToHost,
                                 b->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
            return bcuda(b, e, "lb_batch_set_theta0: max|theta0|");
        for (int j = 0; j < b->count; ++j) {
            if (!(mx[j] > 0.0) || !isfinite(mx[j]))
                return bfail(b, LB_ENONPOS, "lb_batch_set_theta0: theta0 must be finite and > 0");
            int ex = 0;
            frexp(mx[j], &ex);
            b->inst[j].fx_bits = 59 - ex;
            if (b->inst[j].fx_bits > 1000 || b->inst[j].fx_bits < -1000)
                return bfail(b, LB_EINVAL, "lb_batch_set_theta0: theta0 magnitude outside the fixed-point range");
        }
    }
    b->cur = 0;
    for (int j = 0; j < b->count; ++j) {
        lb_ctx &c = b->inst[j];
        c.cur = 0;
        const double *th = theta0 + b->node_off[j];
        const double *gr = grad0 ? grad0 + 2 * b->node_off[j] : b->gradtmp + 2 * b->node_off[j];
        if (!grad0 && (e = lbk::launch_fd4_grad(&c, th, const_cast<double *>(gr))) != cudaSuccess)
            return bcuda(b, e, "lb_batch_set_theta0: fd4");
        if ((e = lbk::launch_init(&c, th, gr, b->d_flag)) != cudaSuccess)
            return bcuda(b, e, "lb_batch_set_theta0: init");
    }
    int flag = 0;
    if ((e = cudaMemcpyAsync(&flag, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return bcuda(b, e, "lb_batch_set_theta0");
    if (flag & 1) return bfail(b, LB_ENONPOS, "lb_batch_set_theta0: theta0 must be finite and > 0");
    if (flag & 2)
        return bfail(b, LB_EINVAL, "lb_batch_set_theta0: a gradient too steep for the fixed-point range");
    b->initialized = true;
    return LB_OK;
}

lb_status lb_batch_step(lb_batch *b, int64_t n)
{
    lbk::NvtxRange nvtx_range("lb_batch_step");
    if (!b) return LB_EINVAL;
    if (n < 0) return bfail(b, LB_EINVAL, "lb_batch_step: n < 0");
    if (!b->initialized) return bfail(b, LB_ESTATE, "lb_batch_step: call lb_batch_set_theta0 first");
    cudaError_t e = run_steps(b, n);
    if (e != cudaSuccess) return bcuda(b, e, "lb_batch_step");
    return LB_OK;
}

lb_status lb_batch_macros(lb_batch *b, double *theta, double *u)
{
    lbk::NvtxRange nvtx_range("lb_batch_macros");
    if (!b) return LB_EINVAL;
    if (!b->initialized) return bfail(b, LB_ESTATE, "lb_batch_macros: call lb_batch_set_theta0 first");
    for (int j = 0; j < b->count; ++j) {
        lb_ctx &c = b->inst[j];
        c.cur = b->cur;
        cudaError_t e = lbk::launch_macros(&c, c.f[b->cur], theta ? theta + b->node_off[j] : nullptr, nullptr,
                                           u ? u + 2 * b->node_off[j] : nullptr, b->d_flag + 1);
        if (e != cudaSuccess) return bcuda(b, e, "lb_batch_macros");
    }
    return LB_OK;
}

lb_status lb_batch_errors(lb_batch *b, const double *theta, const double *u, const double *eth, const double *eu,
                          double *out)
{
    lbk::NvtxRange nvtx_range("lb_batch_errors");
    if (!b || !theta || !eth || !out) return LB_EINVAL;
    if ((u == nullptr) != (eu == nullptr)) return bfail(b, LB_EINVAL, "lb_batch_errors: u and exact_u go together");
    lbk::batch_errors_kernel<<<b->count, lbk::kRedThreads, 0, b->stream>>>(b->d_node_off, theta, u, eth, eu,
                                                                           b->total_nodes, b->d_err);
    cudaError_t e = cudaGetLastError();
    int flag = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, b->d_err, sizeof(double) * 4 * b->count, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&flag, b->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lb_batch_errors");
    if (flag & 4) return bfail(b, LB_ETIMEOUT, "lb_batch_macros: a shared-memory staging wait timed out");
    if (flag) return bfail(b, LB_ENONPOS, "lb_batch_macros saw theta <= 0");
    return LB_OK;
}

lb_status lb_batch_autotune(lb_batch *b, int trial_steps, double *choice)
{
    lbk::NvtxRange nvtx_range("lb_batch_autotune");
    if (!b || trial_steps < 2) return LB_EINVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, LB_ECUDA, "lb_batch_autotune: sync");
    // Candidates: (a) one launch per step per group (byte budget x block
    // size); one instance per group is the naive baseline and never the
    // fastest, so it is left out (lb_batch_set_schedule can still select it);
    // (b) blocked launches: K steps per launch x tile edge (the largest that
    // fits one, two, three or four blocks per SM with a K-node halo, and that
    // edge less 4) x block size.
    struct Cand {
        double budget;
        int threads, K, tile;
    };
    std::vector<Cand> cands;
    for (double bud : {48e6, 96e6, 128e6, 1e18})
        for (int th : {64, 128, 256, 512}) cands.push_back({bud, th, 0, 0});
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess)
        return bfail(b, LB_ECUDA, "lb_batch_autotune: device attribute");
    for (int K : {2, 3, 4, 5, 6, 8, 12})
        for (int per_sm : {1, 2, 3, 4}) {
            const size_t avail = per_sm == 1 ? (size_t)optin : (size_t)optin / per_sm - 1024;
            int edge = 1;  // largest square tile + halo whose buffers fit
            while (lbk::tb_smem_bytes(9, (int)b->elem, edge + 1, edge + 1) <= avail) ++edge;
            // that tile, and one 4 nodes smaller (less work per block)
            for (int tile : {edge - 2 * K, edge - 2 * K - 4}) {
                if (tile < 8) continue;
                for (int th : {256, 512, 1024}) cands.push_back({b->budget, th, K, tile});
            }
        }
    double best = 1e300;
    Cand win = {b->budget, b->threads, b->tb_k, b->tb_tile};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, LB_ECUDA, "lb_batch_autotune: events");
    lb_status st = LB_OK;
    for (const Cand &cd : cands) {
        if (cd.K == 0) {
            if ((st = build_tiles(b, 0, 0, 0)) != LB_OK || (st = build_schedule(b, cd.budget, cd.threads, true)) != LB_OK)
                break;
        } else if ((st = build_tiles(b, cd.K, cd.tile, cd.threads)) != LB_OK) {
            st = LB_OK;  // a tile that does not fit this device is skipped
            continue;
        }
        const int64_t n = cd.K ? (trial_steps + cd.K - 1) / cd.K * cd.K : trial_steps;
        cudaError_t e = run_steps(b, n);  // warm-up: records the graphs, fills L2
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = run_steps(b, n);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            st = bcuda(b, e, "lb_batch_autotune");
            break;
        }
        const double per_step = ms / (double)n;
        if (per_step < best) {
            best = per_step;
            win = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LB_OK) return st;
    b->initialized = false;  // the trials overwrote the state
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, LB_ECUDA, "lb_batch_autotune: sync");
    if (win.K == 0) {
        if ((st = build_tiles(b, 0, 0, 0)) != LB_OK) return st;
        if ((st = build_schedule(b, win.budget, win.threads, true)) != LB_OK) return st;
    } else if ((st = build_tiles(b, win.K, win.tile, win.threads)) != LB_OK) {
        return st;
    }
    if (choice) {
        choice[0] = b->budget;
        choice[1] = win.K ? win.threads : b->threads;
        choice[2] = (double)b->groups.size();
        choice[3] = 1e3 * best;
        choice[4] = win.K;
        choice[5] = win.tile;
    }
    return LB_OK;
}

lb_status lb_batch_set_schedule(lb_batch *b, double budget, int threads, int use_graph)
{
    if (!b || !(threads == 64 || threads == 128 || threads == 256 || threads == 512) || !isfinite(budget))
        return LB_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);  // tables in use by queued launches
    if (e != cudaSuccess) return bcuda(b, e, "lb_batch_set_schedule");
    free_tiles(b);
    return build_schedule(b, budget, threads, use_graph != 0);
}

lb_status lb_batch_set_blocking(lb_batch *b, int steps_per_launch, int tile, int threads, int use_graph)
{
    if (!b) return LB_EINVAL;
    if (steps_per_launch < 0 || steps_per_launch > 64 || (steps_per_launch > 0 && (tile < 1 || tile > 4096)) ||
        (steps_per_launch > 0 && !(threads == 256 || threads == 512 || threads == 1024)))
        return bfail(b, LB_EINVAL, "lb_batch_set_blocking: steps per launch in 0..64, tile >= 1, threads 256, 512 or 1024");
    lb_status st = build_tiles(b, steps_per_launch, tile, threads);
    if (st == LB_OK) b->use_graph = use_graph != 0;
    return st;
}

lb_status lb_batch_schedule(const lb_batch *b, double *info)
{
    if (!b || !info) return LB_EINVAL;
    info[0] = b->budget;
    info[1] = b->tb_k ? b->tb_threads : b->threads;
    info[2] = (double)b->groups.size();
    info[3] = (double)b->total_nodes;
    info[4] = b->tb_k;
    info[5] = b->tb_k ? b->tb_tile : 0;
    info[6] = b->ntiles;
    return LB_OK;
}

const char *lb_batch_last_error(const lb_batch *b) { return b ? b->err.c_str() : "lb_batch: NULL handle"; }

}  // extern "C"
