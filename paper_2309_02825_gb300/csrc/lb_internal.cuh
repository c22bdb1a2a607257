// Internal declarations shared by the C-ABI layer and the kernels.
//
// Storage ("P form"): q arrays, one per discrete velocity, each a padded
// grid [N2][N1][pitch] with x fastest.  The value stored at (i, x) after
// step n is the post-collision f*_i(x, n-1); the pre-collision
// distribution at step n is therefore f_i(x, n) = P_i(x - e_i) (periodic).
// One sweep pulls those values, collides them and writes P_{n+1} aligned,
// so every store is a full aligned vector and only loads are shifted.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <type_traits>

#include "../../include/lb.h"

namespace lbk {

// ---------------------------------------------------------------------------
// Lattices DdQ(1+2d^2) for d = 1..4 in lattice units e_i = c_i / c, in
// the order printed in Eqs. (d1q3), (d2q9) and (d3q19); for d = 4 the
// structure of Eq. (ddqq): rest, +e_p, -e_p, then for each coordinate pair
// (a < b) the four velocities (e_a, e_b) = (1,1), (-1,1), (-1,-1), (1,-1).
// Components beyond d are zero.
// ---------------------------------------------------------------------------
struct D1Q3 {
    static constexpr int D = 1, Q = 3;
    static constexpr int E[Q][4] = {{0, 0, 0, 0}, {1, 0, 0, 0}, {-1, 0, 0, 0}};
};
struct D2Q9 {
    static constexpr int D = 2, Q = 9;
    static constexpr int E[Q][4] = {{0, 0, 0, 0}, {1, 0, 0, 0},  {0, 1, 0, 0},   {-1, 0, 0, 0}, {0, -1, 0, 0},
                                    {1, 1, 0, 0}, {-1, 1, 0, 0}, {-1, -1, 0, 0}, {1, -1, 0, 0}};
};
struct D3Q19 {
    static constexpr int D = 3, Q = 19;
    static constexpr int E[Q][4] = {
        {0, 0, 0, 0},   {1, 0, 0, 0},  {0, 1, 0, 0},   {0, 0, 1, 0},   {-1, 0, 0, 0},  {0, -1, 0, 0}, {0, 0, -1, 0},
        {1, 1, 0, 0},   {-1, 1, 0, 0}, {-1, -1, 0, 0}, {1, -1, 0, 0},  {1, 0, 1, 0},   {-1, 0, 1, 0}, {-1, 0, -1, 0},
        {1, 0, -1, 0},  {0, 1, 1, 0},  {0, -1, 1, 0},  {0, -1, -1, 0}, {0, 1, -1, 0}};
};
struct D4Q33 {
    static constexpr int D = 4, Q = 33;
    static constexpr int E[Q][4] = {
        {0, 0, 0, 0},
        {1, 0, 0, 0},   {0, 1, 0, 0},   {0, 0, 1, 0},   {0, 0, 0, 1},
        {-1, 0, 0, 0},  {0, -1, 0, 0},  {0, 0, -1, 0},  {0, 0, 0, -1},
        {1, 1, 0, 0},   {-1, 1, 0, 0},  {-1, -1, 0, 0}, {1, -1, 0, 0},   // (x1, x2)
        {1, 0, 1, 0},   {-1, 0, 1, 0},  {-1, 0, -1, 0}, {1, 0, -1, 0},   // (x1, x3)
        {1, 0, 0, 1},   {-1, 0, 0, 1},  {-1, 0, 0, -1}, {1, 0, 0, -1},   // (x1, x4)
        {0, 1, 1, 0},   {0, -1, 1, 0},  {0, -1, -1, 0}, {0, 1, -1, 0},   // (x2, x3)
        {0, 1, 0, 1},   {0, -1, 0, 1},  {0, -1, 0, -1}, {0, 1, 0, -1},   // (x2, x4)
        {0, 0, 1, 1},   {0, 0, -1, 1},  {0, 0, -1, -1}, {0, 0, 1, -1}};  // (x3, x4)
};

// Storage vector per thread: 16-byte loads/stores covering V consecutive x.
template <typename T> struct Vec;
template <> struct Vec<double> { using type = double2; static constexpr int V = 2; };
template <> struct Vec<float> { using type = float4; static constexpr int V = 4; };
template <> struct Vec<long long> { using type = longlong2; static constexpr int V = 2; };

// Values of one population a sweep lane holds (consecutive nodes along x).
// One 16-byte vector, except in 4D: with q = 33 populations two-phase
// gathers of one 16-byte vector per population need more registers than
// keep enough warps resident, so the 4D sweep narrows the lane to 8 bytes
// (one int64, two floats); FP64, bound by the FP64 pipe, keeps the vector.
__host__ __device__ inline constexpr int lane_width(int d, int elem_bytes, bool fp64)
{
    return (d == 4 && !fp64) ? 8 / elem_bytes : 16 / elem_bytes;
}
template <class L, typename T> __host__ __device__ constexpr int lane_width()
{
    return lane_width(L::D, (int)sizeof(T), std::is_same<T, double>::value);
}

// Grid geometry of one padded state array.
struct Geom {
    int N0, N1, N2, N3;  // sizes (1 for missing axes)
    int pitch;           // row pitch in elements: N0 rounded up to one 16-byte vector
    int64_t slab;        // pitch*N1*N2: elements per population
    int64_t rows;        // N1*N2*N3
    int seg_per_row;     // ceil(pitch / (32*W)): warp segments per row, W values a lane
    int64_t nseg;        // rows * seg_per_row (one warp per segment)
    unsigned mirror;     // bit a: axis a has mirror walls on nodes 0 and N_a - 1 (else periodic)
    // Flat mapping of the periodic 4D sweep with 8-byte states: the nodes
    // numbered row-major, one per lane, 32 to a warp, running on over row
    // ends.  fseg = its warp count, 0 where rows fill whole warps (or the
    // node count reaches 2^31).
    int64_t fseg;
};

// Index of the velocity e_i with its components on the axes of mask M
// (bit a = axis a) negated: the population a mirror wall normal to those
// axes reflects e_i into.  Every DdQ(1+2d^2) lattice here is closed under
// such reflections.
template <class L> __host__ __device__ constexpr int reflect_pop(int i, int M)
{
    for (int j = 0; j < L::Q; ++j) {
        bool same = true;
        for (int a = 0; a < 4; ++a) {
            const int want = ((M >> a) & 1) ? -L::E[i][a] : L::E[i][a];
            if (L::E[j][a] != want) same = false;
        }
        if (same) return j;
    }
    return -1;
}

// Lanes of a row's last segment may start at or beyond the pitch: they load
// (harmless) values of the next row and never store.  Every state-shaped
// allocation carries this many extra elements so those loads stay inside it.
constexpr int64_t kSlackElems = 128;

// Geometry of a state array: V = elements per 16-byte vector (the pitch
// unit), W = values a sweep lane holds (0: one vector).
inline Geom make_geom(int64_t N0, int64_t N1, int64_t N2, int64_t N3, int V, int W = 0)
{
    if (W <= 0) W = V;
    Geom g;
    g.N0 = (int)N0;
    g.N1 = (int)N1;
    g.N2 = (int)N2;
    g.N3 = (int)N3;
    g.pitch = (int)((N0 + V - 1) / V * V);
    g.rows = N1 * N2 * N3;
    g.slab = (int64_t)g.pitch * g.rows;
    g.seg_per_row = (g.pitch + 32 * W - 1) / (32 * W);
    g.nseg = g.rows * g.seg_per_row;
    g.mirror = 0;
    const int64_t nodes = g.rows * g.N0;
    g.fseg = (g.pitch % (32 * W) != 0 && nodes < (1ll << 31) - 64) ? (nodes + 31) / 32 : 0;
    return g;
}

// Whether a sweep of lattice dimension d with elem-byte states takes the flat
// mapping: measured faster only for 4D 8-byte states (whose row-segment
// gather holds q = 33 vectors and keeps few warps resident), and used only on
// periodic grids.
inline bool sweep_flat(const Geom &g, int d, int elem) { return d == 4 && elem == 8 && g.fseg && !g.mirror; }

// Collision constants (lattice units), precomputed on the host from the
// relaxation set.  With sigma = c_s^2/c^2 = 2 w1 + 4(d-1) wd the
// post-collision distributions are
//   f0*       = c0 theta - 2 k2 sum_a P_aa
//   f(+-e_a)* = k2 P_aa + cA theta +- k1 J_a
//   f(diag)*  = wd theta + sa*sb k3 P_ab
// with k1 = (1-s1)/2, k2 = (1-s2x)/2, k3 = (1-s22)/4,
// c0 = 1 - d s2x sigma + 2 d(d-1) wd and cA = s2x sigma/2 - 2(d-1) wd.
template <typename T> struct Coll {
    T k1, k2, k3, c0, cA, wd;
};

// The same constants in 64-bit fixed point with 64 fractional bits (every
// constant must lie in (-1/2, 1/2): fx_constants_ok); products are rounded
// to nearest.  The rest
// population is formed as theta minus the others, so the collision
// conserves sum f exactly.
struct CollFx {
    long long k1, k2, k3, cA, wd;
};
// The single-grid fixed-point sweep also checks every value it stores
// against |v| < 2^61 and sets *range when one is not (an unstable custom
// relaxation set grows the state until int64 would wrap; FP64 would reach
// Inf/NaN instead).  Moment sums of values below 2^61 that stay below 2^63
// are exact, so a run whose values cross 2^61 is caught at the step it does,
// unless that one step grows them from below 2^61 past 2^63 / q.
struct CollFxR : CollFx {
    int *range;
};
constexpr int kFxCoefBits = 62;  // initialisation and adjoint constants
constexpr int kFxCollBits = 64;  // collision constants (CollFx)

// Recovery constants (Sec. III.C): u_a = ucoef * J_a / theta with
// ucoef = (2 - s1) c; grad_a = gcoef * J_a with gcoef = -s1 / (sigma dx);
// J_a = sum_k e_ka f_k, summed in storage units (both constants carry the
// storage scale, 2^-F for 64-bit fixed point, 1 otherwise).
struct Recov {
    double ucoef, gcoef, theta_ref;
};

// Initialisation constants (first two terms of Eq. (f-feq-o5), closed
// form): f0 = w0 th; f(+-e_a) = w1 th -+ iax * d_a th;
// f(diag e) = wd th - idg * (e . grad th).
struct InitK {
    double w0, w1, wd, iax, idg, theta_ref;
    double fxscale;  // 2^F for 64-bit fixed-point storage, unused otherwise
    // 64-bit fixed point formed in integers: theta -> round(theta 2^F), a
    // gradient component -> round(dx grad 2^F) (gscale = dx 2^F), and the
    // constants w1, wd, iax/dx with kFxCoefBits fraction bits.
    double gscale;
    long long w1k, wdk, iak;
    int fx_bits;  // F
};

}  // namespace lbk

// ---------------------------------------------------------------------------
// Context.
// ---------------------------------------------------------------------------
struct lb_ctx {
    int d = 0, q = 0;
    int64_t N[4] = {1, 1, 1, 1};
    int64_t nodes = 0;
    int precision = LB_FP64;
    double nu = 0, dx = 0, dt = 0, c = 0, eps = 0, cs2 = 0, sigma = 0;
    double s1 = 0, s2x = 0, s22 = 1, w0 = 0, w1 = 0, wd = 0, theta_ref = 0;
    int fx_bits = 0;          // LB_FX64: stored value = round(f * 2^fx_bits)
    double fx_max = 0.0;      // LB_FX64: if > 0, the max |theta0| that fixes fx_bits (a slab's global maximum)
    bool paper = true;        // relaxation set from Theorem 2 (eps-derivatives known)
    cudaStream_t stream = nullptr;
    lbk::Geom geom{};
    size_t elem = 8;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    double *scratch = nullptr;     // reduction partials
    int scratch_blocks = 0;
    double *dout = nullptr;        // small device result area
    int *dflag = nullptr;          // device status flags
    double *gradtmp = nullptr;     // FD gradient when none is supplied
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // recorded sweeps, by starting buffer
    bool initialized = false;
    int64_t step = 0;
    int device = 0;
    uint64_t gen = 0;  // bumped whenever the walls or the viscosity change (recorded launches go stale)
    // temporally blocked sweeps (lb_set_blocking, 2D periodic): tb_k steps per launch, 0 = one sweep per launch
    int tb_k = 0, tb_tile = 0, tb_threads = 0, tb_ntiles = 0, tb_maxw = 0, tb_maxh = 0;
    void *tb_desc = nullptr;   // instance descriptor of the grid (device)
    void *tb_tiles = nullptr;  // tile table (device)
    cudaGraphExec_t tb_graph[2] = {nullptr, nullptr};  // recorded blocked launches, by starting buffer
    std::string err;
};

namespace lbk {

// NVTX range over one ABI call (visible in Nsight timelines; no cost when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host-side derivation shared by every entry point (single grid and batch):
// relaxation set (Theorem 2, Eq. (Bur-Sol), or the caller's), weights
// (Eq. (d1-3-weight)), sigma = c_s^2/c^2 and the collision constants.
// Returns false if a rate leaves (0, 2) or a weight is not finite.
bool derive_params(lb_ctx &c, const lb_relax *rs);
template <typename T> Coll<T> make_coll(const lb_ctx &c);
CollFx make_coll_fx(const lb_ctx *c);  // the same constants in 64-bit fixed point
// True when every fixed-point collision constant of c (k1, k2, k3, cA, wd)
// lies in (-1/2 + 2^-30, 1/2 - 2^-30), the range of the collision's
// split-word product.  Any relaxation rate in (0, 2) gives |k1|, |k2| < 1/2
// and |k3| < 1/4; wd and cA grow with the weights (the paper's set leaves
// the range only for eps above 1.66 in 2D, 0.88 in 3D and 0.61 in 4D).
bool fx_constants_ok(const lb_ctx &c);
// Device flags of a context (ctx->dflag): 0 initialisation, 1 recovery
// (bit 0: theta <= 0 or non-finite, bit 2: a staging wait timed out),
// 2 fixed-point sweep range (CollFxR).
constexpr int kFlagInit = 0, kFlagRecover = 1, kFlagRange = 2;

constexpr int kRedThreads = 256;
constexpr int kRedSlots = 16;  // doubles per block partial (>= 3*(d+1)+1)

// Launchers (lb_kernels.cu).  All enqueue on ctx->stream and return the
// launch error.
cudaError_t launch_fd4_grad(const lb_ctx *c, const double *theta0, double *grad);
cudaError_t launch_init(lb_ctx *c, const double *theta0, const double *grad, int *flag);
cudaError_t launch_sweep(lb_ctx *c, const void *src, void *dst);
// Recovery (lb_recover.cu); flag bit 0: theta <= 0 seen, bit 2: a staging wait timed out.
cudaError_t launch_macros(lb_ctx *c, const void *src, double *theta, double *grad, double *u, int *flag);
cudaError_t launch_sum_state(lb_ctx *c, const void *src, double *out_dev);
// The same on rows row0 .. row0 + nrow - 1 of the grid only (rows = the
// products of all axes but x, slowest last); the recovery's outputs then hold
// those rows only.
cudaError_t launch_sum_state_rows(lb_ctx *c, const void *src, double *out_dev, int64_t row0, int64_t nrow);
cudaError_t launch_macros_rows(lb_ctx *c, const void *src, double *theta, double *grad, double *u, int *flag,
                               int64_t row0, int64_t nrow);
cudaError_t launch_maxabs(lb_ctx *c, const double *x, int64_t n, double *out_dev);
// 64-bit fixed-point path (lb_fx.cu).
cudaError_t launch_sweep_fx(lb_ctx *c, const void *src, void *dst);
cudaError_t launch_norms(lb_ctx *c, const double *theta, const double *u, const double *ex_theta,
                         const double *ex_u, double *out_dev);
// Temporally blocked sweeps of one 2D periodic grid (lb_batch.cu, the batched
// blocked kernel on a batch of one): set up the tile table and descriptor for
// K steps per launch (K = 0 releases them), and launch K steps from src to dst.
// The fixed-point path checks the values it stores (|f| < 2^61) into
// ctx->dflag[kFlagRange].
cudaError_t blocked_setup(lb_ctx *c, int K, int tile, int threads, bool *fits);
cudaError_t blocked_launch(lb_ctx *c, const void *src, void *dst, int K, cudaStream_t s);
void blocked_release(lb_ctx *c);

}  // namespace lbk
