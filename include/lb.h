/*
 * lb.h - C ABI of the GB300 Cole-Hopf fourth-order MRT-LB solver.
 *
 * Method: Chen, Liu, Chai & Shi, "A Cole-Hopf transformation based
 * fourth-order multiple-relaxation-time lattice Boltzmann model for the
 * coupled Burgers' equations" (arXiv:2309.02825).  The coupled Burgers'
 * velocity u is recovered through the Cole-Hopf map u = -2 nu grad(theta) /
 * theta (Eq. (transf)) from theta solving d(theta)/dt = nu lap(theta)
 * (Eq. (eq-theta)), which is advanced by the MRT-LB scheme of Sec. III.A on
 * the DdQ(1+2d^2) lattice (d = 1, 2, 3, 4: D1Q3, D2Q9, D3Q19, D4Q33).
 *
 * Conventions for every call:
 *  - Every call returns an lb_status; nothing aborts or throws across the
 *    ABI.  lb_last_error() gives a message for the last failure.
 *  - Grids are periodic with sizes N[0..d-1] (N[0] along x, the fastest
 *    axis); nodes sit at x_a = j*dx, j = 0..N[a]-1.
 *  - Field arguments are caller-owned DEVICE pointers to contiguous IEEE
 *    double arrays: a scalar field has N[0]*...*N[d-1] entries with x
 *    fastest; a vector field is d such arrays back to back (component a =
 *    axis a first).  The library never frees or retains them past the call.
 *  - The context owns its device state (two distribution buffers and a
 *    small reduction scratch area); they are freed by lb_destroy.
 *  - Work is enqueued on the CUDA stream given to lb_create, in call order.
 *    Calls whose output lands in host memory (lb_set_theta0's positivity
 *    check, lb_sum_theta, lb_reduce) synchronise that stream before they
 *    return; the others are asynchronous.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef LB_H
#define LB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,   /* an argument is out of range or a pointer is NULL */
    LB_ENOMEM = 2,   /* a device allocation failed */
    LB_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    LB_ESTATE = 4,   /* called out of order (e.g. lb_step before lb_set_theta0) */
    LB_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    LB_ENONPOS = 6   /* theta <= 0 or non-finite where Cole-Hopf needs theta > 0 */
} lb_status;

typedef enum {
    LB_FP64 = 0,         /* distributions stored and updated in IEEE double */
    LB_FP32_SHIFTED = 1, /* stored and updated in float as f - w*theta_ref */
    LB_FX64 = 2          /* stored as 64-bit fixed point round(f * 2^F), with F
                            chosen by lb_set_theta0 so that max|theta0| * 2^F <
                            2^59 (sums up to 16 max|theta0| fit); moment
                            sums are exact integer additions, each relaxation
                            product is rounded once (2^-62 relative), and the
                            rest population is theta minus the others, so
                            sum theta is conserved exactly.  Recovery is FP64. */
} lb_precision;

/*
 * Relaxation set (Sec. III.A, Theorem 2).  With paper_set != 0 the fields
 * s1, s2x, s22, w1, wd are ignored and taken from Eq. (Bur-Sol) with
 * eps = nu*dt/dx^2:
 *   s1 = 2/(6 eps + 1), s2x = 24 eps/(6 eps + 1)^2  (s_2 for d = 1, s_21 for
 *   d > 1), s22 = 4/(6 eps + 3), w1 = 1/6 - (d-1) eps/3, wd = eps/6
 *   (w1 = 1/6 and no wd for d = 1).
 * Otherwise they are used as given (each rate must lie in (0, 2), Sec. III.A);
 * w0 = 1 - 2d w1 - 2d(d-1) wd (Eq. (d1-3-weight)).  Weights need not be
 * positive.  theta_ref is the reference value of LB_FP32_SHIFTED storage
 * (typically the mean of theta0); it is ignored for LB_FP64.
 */
typedef struct {
    int paper_set;
    double s1, s2x, s22, w1, wd;
    double theta_ref;
} lb_relax;

/*
 * Create a solver context.
 *   d        1, 2, 3 or 4.
 *   N        host array of d sizes, each >= 1 (a size of 1 makes that axis
 *            trivially periodic); N[0] <= 2^24, product <= 2^31.
 *   nu, dx, dt  viscosity, lattice spacing, time step (all > 0, finite);
 *            c = dx/dt is the lattice speed.
 *   rs       relaxation set (NULL = paper set, theta_ref = 0).
 *   precision  LB_FP64, LB_FP32_SHIFTED or LB_FX64.
 *   stream   a cudaStream_t (NULL = the legacy default stream).
 *   out      receives the context; set to NULL on failure.
 * Allocates 2*q*pitch*N[1]*N[2] distribution values on the current device.
 * LB_FX64 holds the collision constants k1 = (1-s1)/2, k2 = (1-s2x)/2,
 * k3 = (1-s22)/4, cA = s2x sigma/2 - 2(d-1) wd and wd with 64 fraction bits
 * and needs each inside (-1/2, 1/2) (by a margin of 2^-30): k1, k2, k3
 * always are; the paper's set keeps cA and wd inside for eps below 1.66
 * (d = 2), 0.88 (d = 3), 0.61 (d = 4) and for every eps when d = 1.
 * Errors: LB_EINVAL (also a constant outside that range for LB_FX64),
 * LB_ENOMEM, LB_ECUDA.
 */
lb_status lb_create(int d, const int64_t *N, double nu, double dx, double dt,
                    const lb_relax *rs, int precision, void *stream, lb_ctx **out);

/* Release the context and its device memory (after synchronising its stream). NULL is a no-op. */
lb_status lb_destroy(lb_ctx *ctx);

/*
 * Parameters in use, written to out[0..14] (host):
 *   eps, c, cs2 (= c_s^2, Eq. (conseved-moment)), s1, s2x, s22, w0, w1, wd,
 *   nu, dx, dt, q, theta_ref, F (LB_FX64 fraction bits; 0 before
 *   lb_set_theta0 and for the other precisions).
 */
lb_status lb_get_params(const lb_ctx *ctx, double *out);

/*
 * Boundary kind of one axis.  The paper's Examples 2-4 are periodic; its
 * Example 1 (Sec. V) prescribes u = 0 at both ends of [0, 1], which under
 * the Cole-Hopf transformation u = -2 nu grad theta / theta is the
 * homogeneous Neumann condition d theta / dn = 0.  The paper does not state
 * how its LB scheme imposes it; LB_MIRROR does it by specular reflection:
 * the walls sit on the first and last node of the axis (N_a nodes span
 * (N_a - 1) dx), and a population pulled from beyond a wall is read at the
 * mirror image of its source node with its wall-normal velocity component
 * negated.  The result equals, node for node, the periodic scheme on the
 * grid doubled by even reflection across the walls, so the wall adds no
 * error of its own (fourth order is kept), the normal component of u (and of
 * grad theta) vanishes on wall nodes, and sum theta weighted 1/2 per wall a
 * node lies on is conserved (exactly for LB_FX64).
 */
typedef enum {
    LB_PERIODIC = 0,
    LB_MIRROR = 1
} lb_boundary;

/*
 * Set the boundary kind of each axis: kind is a host array of d values
 * (LB_PERIODIC or LB_MIRROR; a new context is periodic on every axis).  A
 * mirror axis needs N_a >= 3.  Synchronises the stream, drops recorded
 * sweeps and leaves the context uninitialised: call lb_set_theta0 next.
 * The initialisation reads theta0 and grad theta0 on the doubled grid:
 * theta0 even across each wall, grad theta0's wall-normal component odd
 * (so it is taken as zero on the wall nodes whatever the caller passes).
 * lb_sum_theta returns the wall-weighted sum on such grids; the discrete
 * adjoint (lb_adjoint.h) differentiates the walled scheme too.
 * Errors: LB_EINVAL (NULL kind, unknown kind, N_a < 3 on a mirror axis),
 * LB_ECUDA.
 */
lb_status lb_set_boundary(lb_ctx *ctx, const int *kind);

/*
 * Change the viscosity nu of a context in place (eps = nu dt / dx^2; dx and
 * dt are kept).  With the paper's relaxation set the rates and weights are
 * re-derived from Eq. (Bur-Sol) at the new eps; a caller's set is kept as
 * given.  The stored state is kept (the next lb_step continues from it with
 * the new collision), nothing is allocated, and recorded sweeps are dropped
 * after synchronising the stream.  An adjoint workspace whose forward pass
 * predates the change refuses reverse steps (LB_ESTATE) until
 * lb_adjoint_forward runs again.
 * Errors: LB_EINVAL (nu not finite and > 0, a rate leaving (0, 2), or for
 * LB_FX64 a collision constant leaving (-1/2, 1/2), as in lb_create),
 * LB_ECUDA.
 */
lb_status lb_set_viscosity(lb_ctx *ctx, double nu);

/* The boundary kind of each axis, written to kind[0..d-1] (host). */
lb_status lb_get_boundary(const lb_ctx *ctx, int *kind);

/*
 * Initialise the distributions from theta0 (Sec. IV: the first two terms of
 * Eq. (f-feq-o5)):  f_i(x, 0) = w_i theta0 - dt [M^-1 S^-1 M Dbar (w theta0)]_i
 * with Dbar = diag(c_i . grad).
 *   theta0       device, scalar field, every value finite and > 0.
 *   grad_theta0  device, vector field (d*nodes) holding grad theta0, or NULL
 *                to use a fourth-order central difference of theta0.
 * Resets the step counter to 0.  For LB_FX64 it also fixes the fixed-point
 * scale F from max|theta0|.  Synchronises the stream.
 * Errors: LB_EINVAL (NULL theta0; for LB_FX64 also an initial value beyond
 * 4 max|theta0|, i.e. a gradient too steep for the fixed-point range),
 * LB_ENONPOS (theta0 <= 0 or non-finite
 * somewhere, or a non-finite gradient; the state is then left uninitialised),
 * LB_ECUDA.
 */
lb_status lb_set_theta0(lb_ctx *ctx, const double *theta0, const double *grad_theta0);

/*
 * Advance nsteps >= 0 time steps of Eq. (distribution-f): at every node the
 * pre-collision f is pulled from the neighbours (streaming), relaxed in
 * moment space (m* = m - S (m - m^eq), m^eq = M w theta) and stored.
 * Asynchronous.  For LB_FX64 every stored value is checked against
 * |f| < 2^61 (reported by lb_macros, lb_sum_theta or lb_check).
 * Errors: LB_EINVAL (nsteps < 0), LB_ESTATE (no
 * lb_set_theta0 yet, or a reported timeout or range overflow since), LB_ECUDA.
 */
lb_status lb_step(lb_ctx *ctx, int64_t nsteps);

/*
 * Temporally blocked sweeps (periodic 2D grids).  The sweep of lb_step reads
 * and writes the whole state every step, so it is bound by HBM bandwidth.
 * With blocking, each launch advances K steps: a block loads one tile of
 * the grid with a K-node periodic halo into shared memory, runs the same
 * pull + collide K times there (one shared buffer, updated in place: steps
 * alternate between pulling from the neighbours' slots and updating a
 * node's own slots, and each node reads exactly the slots it writes) and
 * stores the tile, so HBM is read and written once per K steps; the halo
 * nodes are recomputed.  Results are bit-identical to lb_step's one sweep per
 * launch.  For LB_FX64 the range check (|f| < 2^61) covers the values
 * stored at the end of every launch.
 *   steps_per_launch  K in 1..64, or 0 for one sweep per launch (default).
 *   tile     each axis of N nodes is cut into ceil(N / tile) near-equal tiles;
 *            the largest tile plus its halo, 9 values per node, must fit the
 *            device's shared memory per block.
 *   threads  256, 512 or 1024 per block.
 * Synchronises the stream; keeps the state.  lb_set_boundary with a mirror
 * axis returns the context to one sweep per launch.
 * Errors: LB_EINVAL (out of range, d != 2, walls, or a tile too large), LB_ECUDA.
 */
lb_status lb_set_blocking(lb_ctx *ctx, int steps_per_launch, int tile, int threads);

/* Current blocking, info[0..3] (host): {steps per launch (0: none), tile, threads, tiles}. */
lb_status lb_get_blocking(const lb_ctx *ctx, int *info);

/*
 * Times about trial_steps steps (rounded up to whole launches) for one sweep
 * per launch and for blocked sweeps (K = 2, 3, 4, 5, 6, 8, 12 x the largest
 * square tile that fits one to four blocks per SM and that tile less 4 nodes
 * x 256, 512, 1024 threads) on this
 * grid and keeps the fastest (lb_set_blocking).  The trials overwrite the
 * state: call lb_set_theta0 afterwards.  A grid that blocking does not cover
 * (d != 2, walls) keeps one sweep per launch.  choice (host, may be NULL)
 * receives {steps per launch (0: one sweep per launch), tile, threads,
 * microseconds per step of the winner}.  Synchronises the stream.
 * Errors: LB_EINVAL, LB_ECUDA.
 */
lb_status lb_autotune(lb_ctx *ctx, int trial_steps, double *choice);

/* Number of steps taken since the last lb_set_theta0 (host, no sync). */
lb_status lb_get_step(const lb_ctx *ctx, int64_t *nsteps);

/*
 * Macroscopic recovery at the current time from the pre-collision f
 * (Sec. III.C):
 *   theta = sum_k f_k,
 *   grad theta = -s1 sum_k c_k f^ne_k / (dt c_s^2)   (Eq. (nabla-theta)),
 *   u_a = (2 - s1) sum_k c_ka f^ne_k / sum_k f_k     (Eq. (ui-compute)).
 * All three are computed in FP64 (also for LB_FP32_SHIFTED).  Each block
 * stages its row segment of every population, with the one-node x-halo, in
 * shared memory by bulk asynchronous copies (TMA) completing on an mbarrier.
 * Any output pointer may be NULL to skip it.  Device outputs: theta (nodes),
 * grad_theta and u (d*nodes).  The call synchronises the stream and reports
 * what the device saw since the last report: LB_ENONPOS for a node with
 * theta <= 0 or non-finite, LB_ETIMEOUT for a staging wait that gave up
 * (bounded at 1 s; its tile may be incomplete, so the outputs are not to be
 * used and the context refuses lb_step / lb_macros until lb_set_theta0 or
 * lb_load_state sets a state again), and for LB_FX64 LB_EINVAL when a sweep
 * stored a value with |f| >= 2^61 (an unstable run: FP64 would overflow to
 * non-finite values; the context is likewise left without a state).  While
 * the stream is being captured into a CUDA graph the call only enqueues the
 * kernel; the flags are then reported by lb_check, lb_sum_theta or lb_reduce.
 * Errors: LB_ESTATE, LB_ENONPOS, LB_ETIMEOUT, LB_EINVAL, LB_ECUDA.
 */
lb_status lb_macros(lb_ctx *ctx, double *theta, double *grad_theta, double *u);

/*
 * Synchronise the stream and report (then clear) the device-side flags of
 * the work enqueued so far, as lb_macros does: LB_ENONPOS, LB_ETIMEOUT, or
 * LB_EINVAL for a fixed-point range overflow of a sweep (LB_FX64).  LB_OK
 * when none is set.  For callers that step without recovering, and after
 * a captured graph ran.  Errors: as listed, LB_ECUDA.
 */
lb_status lb_check(lb_ctx *ctx);

/*
 * Conserved total sum_x theta(x) = sum over nodes and populations of f,
 * accumulated in FP64 (exactly conserved up to rounding on a periodic grid).
 * out: host, 1 value.  Synchronises the stream.  For LB_FX64 it also reports
 * (LB_EINVAL) a sweep that stored a value with |f| >= 2^61 since the last
 * report.  Errors: LB_ESTATE, LB_EINVAL, LB_ECUDA.
 */
lb_status lb_sum_theta(lb_ctx *ctx, double *out);

/*
 * Error norms of the recovered fields against reference fields (Sec. IV,
 * RMSE per variable).  Device inputs: theta and exact_theta (nodes), u and
 * exact_u (d*nodes; both NULL to skip the velocity).  Host output out, with
 * V = 1 + d variables (theta, u_1, ..., u_d) and for variable v:
 *   out[3v+0] = RMSE   = sqrt(sum (psi - psi*)^2 / nodes)
 *   out[3v+1] = Linf   = max |psi - psi*|
 *   out[3v+2] = rel L2 = sqrt(sum (psi - psi*)^2 / sum psi*^2)
 * and out[3V] = sum theta.  FP64 with a deterministic two-level reduction
 * (warp shuffles, then a fixed-order pass over per-block partials held in
 * the context's scratch area).  Synchronises the stream.
 * Errors: LB_EINVAL, LB_ENONPOS (a previous lb_macros, run inside a stream
 * capture, saw theta <= 0), LB_ETIMEOUT (likewise for a staging wait), LB_ECUDA.
 */
lb_status lb_reduce(lb_ctx *ctx, const double *theta, const double *u,
                    const double *exact_theta, const double *exact_u, double *out);

/*
 * Error norms without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc -- a host application
 * whose framework owns all device memory through its own caching allocator,
 * a service held to a device-memory budget fixed up front, or code where the
 * implicit synchronisation of an allocation is not allowed -- and that
 * therefore have no context (lb_create allocates).
 * Same inputs and results as lb_reduce, with device pointers throughout:
 *   d            1, 2 or 3;  nodes: number of nodes, 1 .. 2^31.
 *   theta, exact_theta  device, nodes values each; u, exact_u device,
 *                d*nodes values each, or both NULL.
 *   out          DEVICE pointer to 3(d+1)+1 doubles, written in lb_reduce's
 *                layout (RMSE, Linf, rel L2 per variable, then sum theta).
 *   stream       a cudaStream_t (NULL = legacy default stream); asynchronous.
 * Scratch: a file-scope __device__ array of 131,200 bytes (1024 partial
 * rows of 16 doubles plus one row of raw sums) that every GPU loading this
 * library holds until the process exits.  Each call made outside a stream
 * capture looks up that array's device address (cudaGetSymbolAddress) with
 * the device current, so an address from before a cudaDeviceReset is never
 * reused; a call inside a capture uses the address of an earlier call on
 * that device, so make a first call before any stream capture (and again
 * after a cudaDeviceReset).  All pointers must be on the current device.  Each call
 * overwrites every row it reads, so nothing needs clearing between calls,
 * but all calls share the one array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be ordered by the caller.
 * Errors: LB_EINVAL (d outside 1..3, nodes outside 1..2^31, a NULL input or
 * out, u without exact_u), LB_ECUDA (address lookup or launch failed); no
 * message is recorded for lb_last_error.
 */
lb_status lb_reduce_static(int d, int64_t nodes, const double *theta, const double *u,
                           const double *exact_theta, const double *exact_u, double *out, void *stream);

/*
 * Copy the raw distribution state to/from a caller buffer (checkpointing).
 * The state is q arrays in the context's padded layout (lb_state_layout):
 * value (i, x, y, z) sits at element i*slab + (z*N[1] + y)*pitch + x.
 * Values are stored after collision and before streaming: the pre-collision
 * distribution at the current step n is f_i(x, n) = state_i(x - e_i)
 * (periodic).  For LB_FP32_SHIFTED the stored value is f - w_i*theta_ref;
 * for LB_FX64 it is round(f * 2^F) as int64 (F from lb_get_params; a state
 * loaded into another context is read with that context's F).
 * Padding entries (x >= N[0]) are ignored.  buf is a device pointer of
 * q*slab*elem_bytes bytes.  lb_load_state sets the step counter to `step`.
 */
lb_status lb_state_layout(const lb_ctx *ctx, int64_t *pitch, int64_t *slab, int64_t *elem_bytes);
lb_status lb_save_state(lb_ctx *ctx, void *buf);
lb_status lb_load_state(lb_ctx *ctx, const void *buf, int64_t step);

/*
 * Self-test of the bounded waits used by the staged recovery: runs one block
 * whose mbarrier phase is never completed and returns LB_ETIMEOUT once the
 * bounded wait gives up after limit_s seconds (0 < limit_s <= 10), leaving
 * the device usable; LB_OK would mean the wait was not bounded.  waited_s
 * (host, may be NULL) receives the kernel's duration.  No paper counterpart.
 */
lb_status lb_selftest_staging_timeout(double limit_s, void *stream, double *waited_s);

/*
 * Self-test of the integer -> FP64 conversions (round to nearest, ties to
 * even, assembled from the IEEE 754 binary64 encoding on the integer pipes)
 * that the fixed-point reverse pass uses for its exact 128-bit sums.  For
 * i < n: out128[i] = the 128-bit integer hi[i] * 2^64 + lo[i] (hi signed,
 * lo unsigned) converted, out64[i] = lo[i] read as a signed 64-bit integer,
 * converted.  All four arrays are caller-owned device arrays of n entries;
 * the call is ordered on `stream` and synchronises it.  LB_EINVAL for n < 0
 * or a NULL array with n > 0.  No paper counterpart.
 */
lb_status lb_selftest_int_to_f64(const long long *hi, const unsigned long long *lo, int64_t n, double *out128,
                                 double *out64, void *stream);

/*
 * Self-test of the fixed-point collision product: for i < n,
 * out_split[i] = the split-word product the LB_FX64 collisions use and
 * out_wide[i] = the same value from a 128-bit product, both
 * floor((a[i] k[i] + 2^63) / 2^64), i.e. a[i] k[i] / 2^64 rounded to nearest
 * with ties upward (k[i] a constant with 64 fraction bits).  The split form
 * is exact for |k[i]| <= 2^63 - 2^34 (the range lb_create admits for the
 * constants) and |a[i]| < 2^63 - 2^31 (the fields stay far below 2^61).  All five arrays are caller-owned device arrays
 * of n entries; the call is ordered on `stream` and synchronises it.
 * LB_EINVAL for n < 0 or a NULL array with n > 0.  No paper counterpart.
 */
lb_status lb_selftest_mulfx(const long long *a, const long long *k, int64_t n, long long *out_split,
                            long long *out_wide, void *stream);

/* Message for the last failing call on ctx (or of lb_create, with ctx == NULL). */
const char *lb_last_error(const lb_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
