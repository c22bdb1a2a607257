/*
 * lb_slab.h - one part of a grid cut into slabs along its slowest axis, for
 * running one grid on several GPUs (one process and one part per GPU).
 *
 * The step of Eq. (distribution-f) streams every population one node along
 * its velocity, so a cut across the slowest axis (axis d-1) is crossed, in
 * each direction, by the populations whose velocity has a +1 (or -1)
 * component on that axis: 3 of 9 for D2Q9, 5 of 19 for D3Q19, 7 of 33 for
 * D4Q33.  A part holds its own layers of the grid (a layer = every node with
 * one coordinate on the slowest axis) plus one ghost layer on each side, in
 * an ordinary context (lb.h) whose sweep is unchanged.  Before every sweep
 * the layers next to each cut trade those populations: the stored
 * post-collision values (lb.h's P form) of the first and last owned layers
 * go to the neighbouring parts' ghost layers, and the sweep then pulls them
 * across the cut exactly as a single grid would.  Every owned node therefore
 * sees the inputs it would see in the whole grid, and the result equals the
 * single-grid solve bit for bit (also for LB_FX64, where every part uses the
 * fixed-point scale of the whole grid).
 *
 * The exchange itself is the caller's: pack into two device buffers, move
 * them to the neighbours (NCCL send/recv between GPUs, a device copy between
 * parts on one GPU), unpack the two received buffers, then lb_slab_step.
 * Parts are numbered 0 .. nparts-1 along the slowest axis, periodically:
 * part p sends its "up" buffer to part (p+1) mod nparts and its "down"
 * buffer to part (p-1) mod nparts.  Bytes per cut and direction per step:
 * (crossing populations) x (one layer: N0 padded to 16 bytes, times the
 * middle axes) x the storage size.
 * Conventions are those of lb.h (status codes, stream order, device
 * pointers).  The paper runs one grid on one machine; slabs are a scaling
 * feature of this library.
 */
#ifndef LB_SLAB_H
#define LB_SLAB_H

#include <stdint.h>

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_slab lb_slab;

/*
 * Part `part` (0 .. nparts-1) of the periodic grid N[0..d-1] (d = 2, 3 or 4),
 * cut along axis d-1 into nparts slabs of N[d-1]/nparts layers (the first
 * N[d-1] mod nparts parts take one more).  Every part needs at least one
 * layer.  nu, dx, dt, rs, precision and stream as for lb_create.
 * Allocates the part's context: its layers plus two ghost layers.
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA.
 */
lb_status lb_slab_create(int d, const int64_t *N, int part, int nparts, double nu, double dx, double dt,
                         const lb_relax *rs, int precision, void *stream, lb_slab **out);
lb_status lb_slab_destroy(lb_slab *s);

/*
 * Facts of the part (host, 6 values): {first owned layer (global index),
 * owned layers, values per pack buffer, bytes per value, crossing
 * populations per direction, nodes per layer}.
 */
lb_status lb_slab_info(const lb_slab *s, int64_t *info);

/* The part's context (its layers and ghost layers), e.g. for lb_get_params or
 * lb_save_state; lb_step on it directly skips the exchange and is wrong. */
lb_ctx *lb_slab_ctx(lb_slab *s);

/*
 * Initialise the part as lb_set_theta0 does on the whole grid.
 *   theta0  device, the part's owned layers plus one layer on each side from
 *           the neighbouring parts (periodic): (owned + 2) layers of N0 x ...
 *           values, x fastest, lowest layer first.
 *   grad    device, the same layers of grad theta0 (d components, each a
 *           field of that shape); required (a difference stencil would need
 *           layers beyond the ghost layers).
 *   max_abs_theta0  max |theta0| over the whole grid (for LB_FX64: the
 *           fixed-point scale every part must share; ignored otherwise).
 * Synchronises the stream.  Errors as lb_set_theta0, and LB_EINVAL for a
 * NULL grad or a part whose max |theta0| exceeds max_abs_theta0.
 */
lb_status lb_slab_set_theta0(lb_slab *s, const double *theta0, const double *grad, double max_abs_theta0);

/*
 * Pack the populations that leave the part: send_up (to part p+1) receives
 * the velocities with a +1 component on the slowest axis from the last owned
 * layer, send_down (to part p-1) those with -1 from the first owned layer;
 * each buffer holds info[2] values (device, storage type of the precision,
 * 16-byte aligned; LB_EINVAL otherwise).  One launch moves both directions.
 * Asynchronous.  Errors: LB_ESTATE (no state), LB_EINVAL, LB_ECUDA.
 */
lb_status lb_slab_pack(lb_slab *s, void *send_down, void *send_up);

/*
 * Unpack what the neighbours sent: recv_down (part p-1's send_up) into the
 * lower ghost layer, recv_up (part p+1's send_down) into the upper one
 * (16-byte aligned buffers, one launch).  Asynchronous.  Errors: LB_ESTATE,
 * LB_EINVAL, LB_ECUDA.
 */
lb_status lb_slab_unpack(lb_slab *s, const void *recv_down, const void *recv_up);

/*
 * One sweep of the part (lb_step on its context).  LB_ESTATE unless
 * lb_slab_unpack ran since the last sweep (or initialisation): a sweep on
 * stale ghost layers would pull wrong values across the cuts.
 */
lb_status lb_slab_step(lb_slab *s);

/*
 * Recovery (as lb_macros) on the owned layers only, after an exchange
 * (lb_slab_unpack) since the last sweep; outputs (device, may be NULL) hold
 * the owned layers: theta owned x layer nodes, grad and u d times that.
 * Reads back the part's device flags (as lb_macros).  Errors: LB_ESTATE,
 * LB_ENONPOS, LB_ETIMEOUT, LB_EINVAL, LB_ECUDA.
 */
lb_status lb_slab_macros(lb_slab *s, double *theta, double *grad, double *u);

/*
 * Sum of theta over the owned layers (host, 1 value); the whole grid's
 * total is the sum over parts.  Synchronises the stream.
 */
lb_status lb_slab_sum_theta(lb_slab *s, double *out);

#ifdef __cplusplus
}
#endif

#endif /* LB_SLAB_H */
