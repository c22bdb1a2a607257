/*
 * lb_batch.h - many independent 2D periodic MRT-LB instances advanced together.
 *
 * Each instance is a separate D2Q9 problem of Sec. III.A (its own N, nu, dx,
 * dt and relaxation set of Theorem 2, Eq. (Bur-Sol)); the paper runs one
 * problem at a time, so batching is a throughput feature of this library.
 * Conventions are those of lb.h (status codes, caller-owned device arrays,
 * stream order).  Fields of all instances are concatenated in instance
 * order: instance j contributes N0_j*N1_j values (x fastest) to a scalar
 * array and 2*N0_j*N1_j (x component first) to a vector array; offsets are
 * the prefix sums of N0_j*N1_j.
 *
 * Scheduling, two kinds:
 *  - one launch per step: instances are bin-packed (largest first) into
 *    groups whose two state buffers fit a byte budget chosen to stay
 *    resident in L2; a group runs all requested steps back to back (each
 *    block of a launch belongs to one instance);
 *  - blocked (lb_batch_set_blocking): each launch advances every instance K
 *    steps.  A block loads one tile of one instance with a K-node periodic
 *    halo into shared memory, runs K steps there (the halo shrinking by one
 *    node per step) and stores the tile, so HBM is read and written once per
 *    K steps instead of every step.  Blocks never wait on one another.
 * Either way the launches are recorded once into CUDA graphs and replayed,
 * and every instance evolves bit for bit as the same grid would alone.
 * lb_batch_autotune times both kinds (budgets, block sizes, steps per
 * launch, tile sizes) on the caller's batch and keeps the fastest.
 */
#ifndef LB_BATCH_H
#define LB_BATCH_H

#include <stdint.h>

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_batch lb_batch;

/*
 * Create a batch of `count` (1..65536) 2D instances.
 *   N     host, 2*count sizes (N0_j, N1_j), each in [1, 2^16].
 *   nu, dx, dt  host, count values each (> 0, finite).
 *   rs    host, count relaxation sets, or NULL for Eq. (Bur-Sol) everywhere
 *         (theta_ref then 0 for every instance; see lb_batch_set_theta_ref).
 *   precision  LB_FP32_SHIFTED, LB_FP64 or LB_FX64 (64-bit fixed point as in lb.h,
 *            each instance scaled by its own max|theta0| at lb_batch_set_theta0,
 *            so an instance evolves bit for bit as the same grid would alone).
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Allocates two state buffers for all instances plus small tables.
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA.
 */
lb_status lb_batch_create(int count, const int64_t *N, const double *nu, const double *dx, const double *dt,
                          const lb_relax *rs, int precision, void *stream, lb_batch **out);

lb_status lb_batch_destroy(lb_batch *b);

/* FP32-shifted reference values, host array of count (default: from rs, else 0). */
lb_status lb_batch_set_theta_ref(lb_batch *b, const double *theta_ref);

/*
 * Initialise every instance as lb_set_theta0 does (Sec. IV, Eq. (f-feq-o5)).
 *   theta0  device, concatenated scalar fields (all > 0).
 *   grad0   device, concatenated vector fields, or NULL for fourth-order
 *           central differences.
 * Synchronises the stream.  Errors: LB_EINVAL, LB_ENONPOS, LB_ECUDA.
 */
lb_status lb_batch_set_theta0(lb_batch *b, const double *theta0, const double *grad0);

/* Advance every instance nsteps (Eq. (distribution-f)); asynchronous. */
lb_status lb_batch_step(lb_batch *b, int64_t nsteps);

/*
 * Recovery for every instance (Sec. III.C), FP64.  theta: device,
 * concatenated scalars; u: device, concatenated vectors; either may be NULL.
 */
lb_status lb_batch_macros(lb_batch *b, double *theta, double *u);

/*
 * Per-instance error norms against concatenated reference fields:
 * out (host) receives 4 values per instance: RMSE(theta), RMSE(|u|) (root of
 * the mean over nodes of the squared error summed over both components),
 * Linf(theta), Linf(u components).  FP64.  Synchronises the stream.
 */
lb_status lb_batch_errors(lb_batch *b, const double *theta, const double *u, const double *exact_theta,
                          const double *exact_u, double *out);

/*
 * Autotuner: times about `trial_steps` steps (rounded up to whole launches)
 * for each candidate on this batch's real sizes and keeps the fastest:
 *  - one launch per step: group byte budget 48, 96, 128 MB or all instances
 *    in one group, x 64, 128, 256 or 512 threads per block;
 *  - blocked: K = 2, 4, 6, 8 or 12 steps per launch x the largest square tile
 *    whose buffer (with the K-node halo) fits one, two, three or four blocks
 *    per SM x 256, 512 or 1024 threads per block.
 * Must be called before lb_batch_set_theta0 (it overwrites the state).
 * choice (host, may be NULL) receives {budget_bytes, threads_per_block,
 * groups, microseconds per step of the winner, steps per launch (0: one
 * launch per step), tile edge (0 likewise)}.  Synchronises the stream.
 */
lb_status lb_batch_autotune(lb_batch *b, int trial_steps, double *choice);

/*
 * Blocked schedule (see the scheduling note above): steps_per_launch K in
 * 1..64 steps per launch; each instance axis of N nodes is cut into
 * ceil(N / tile) near-equal tiles; threads 256, 512 or 1024 per block;
 * use_graph as for lb_batch_set_schedule.  K = 0 returns to one launch per
 * step.  A final launch of fewer than K steps covers a remainder.  Keeps the
 * state.  Errors: LB_EINVAL (out of range, or the largest tile plus its halo
 * needs more shared memory per block than the device has), LB_ECUDA.
 */
lb_status lb_batch_set_blocking(lb_batch *b, int steps_per_launch, int tile, int threads, int use_graph);

/*
 * Set a one-launch-per-step schedule explicitly (leaving blocked launches):
 * budget_bytes <= 0 puts every instance in its own group (one launch per
 * instance per step), a budget above the total state puts all instances in
 * one group (one launch per step); threads is 64, 128, 256 or 512;
 * use_graph = 0 launches every step directly instead of replaying recorded
 * graphs.  Keeps the state.
 */
lb_status lb_batch_set_schedule(lb_batch *b, double budget_bytes, int threads, int use_graph);

/* Current schedule (host, 7 values): {budget_bytes, threads_per_block, groups, total nodes, steps per launch
 * (0: one launch per step), tile edge, tiles}. */
lb_status lb_batch_schedule(const lb_batch *b, double *info);

const char *lb_batch_last_error(const lb_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LB_BATCH_H */
