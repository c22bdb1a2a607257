/*
 * lb_adjoint.h - discrete adjoint of the MRT-LB forward map.
 *
 * Forward map of a context (lb.h): theta0 -> f_0 by Sec. IV's
 * initialisation (first two terms of Eq. (f-feq-o5)) with grad theta0 taken
 * as the fourth-order central difference of theta0 (so the map depends on
 * theta0 alone), T steps of Eq. (distribution-f), and u(T) by
 * Eq. (ui-compute).  The paper has no adjoint; this computes exact
 * gradients of any loss L(u(T), theta(T)) given dL/du and dL/dtheta:
 *   dL/dtheta0 (one value per node) and dL/dnu (through eps = nu dt/dx^2 and
 *   the relaxation set of Theorem 2, Eq. (Bur-Sol); dx and dt fixed).
 * Reverse step: phi_n(x) = K^T [phi_{n+1}(x + e_i)_i]_i (reversed streaming,
 * transposed collision; across a mirror wall the transpose of the reflected
 * pull, which gathers the reflected populations), plus the eps-derivative term
 * lambda_{n+1} . (dK/deps) f_n(x), which needs the forward states f_n: they
 * are kept as checkpoints every C steps and recomputed one segment at a
 * time (C = ceil(sqrt(T)) stores about 2 sqrt(T) states).
 * All calls are stream-ordered on the context's stream.
 */
#ifndef LB_ADJOINT_H
#define LB_ADJOINT_H

#include <stdint.h>

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_adj lb_adj;

/*
 * Adjoint workspace for `ctx` (any precision; d = 1, 2, 3; periodic axes or
 * mirror walls, lb_set_boundary).
 * The forward states are read in their storage type.  The reverse pass
 * computes in FP64 for LB_FP64 contexts, in FP32 for LB_FP32_SHIFTED contexts
 * (whose forward map is FP32-accurate), and for LB_FX64 contexts in 64-bit
 * fixed point: the adjoint field is held as round(phi 2^G), G chosen from
 * the seed so that max|phi_T| 2^G < 2^56, K^T is formed from exact integer
 * sums and rounded 62-bit products, and the dL/dnu term from exact 128-bit
 * dot products (FP64 instead when the collision constants are too large for
 * that range: see lb_adjoint.cu).
 * The seed, the initialisation adjoint and the dL/dnu accumulation are FP64
 * always.
 *   T        forward steps (>= 1).
 *   C        checkpoint interval, 1 <= C <= T, or 0 for ceil(sqrt(T)).
 *   want_nu  nonzero to also compute dL/dnu (needs the paper's relaxation
 *            set; keeps checkpoints and recomputes segments); zero computes
 *            dL/dtheta0 only and keeps no forward states.
 * Allocates ceil(T/C) + 2C state copies (want_nu): the checkpoints and two
 * segment buffers, so that the recomputation of one segment runs beside the
 * reverse steps of the next; the second segment buffer is left out (and
 * segments recomputed one at a time) when there is one segment or the device
 * has no room for it, which lb_adjoint_info's byte count shows.  Also two
 * adjoint fields (8 bytes per value, 4 for LB_FP32_SHIFTED).  The context
 * must outlive the workspace.
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA.
 */
lb_status lb_adjoint_create(lb_ctx *ctx, int64_t T, int64_t C, int want_nu, lb_adj **out);
lb_status lb_adjoint_destroy(lb_adj *a);

/*
 * Forward pass: lb_set_theta0(ctx, theta0, NULL), T steps with checkpoints,
 * then the recovery at T into u (device, d*nodes, may be NULL) and theta
 * (device, nodes, may be NULL).  Errors as lb_set_theta0 / lb_step.
 */
lb_status lb_adjoint_forward(lb_adj *a, const double *theta0, double *theta, double *u);

/*
 * Start the reverse pass from the loss's derivatives at T: seeds
 * phi_T = dL/df_T through Eq. (ui-compute) for u and through
 * theta = sum_k f_k (Eq. (conseved-moment)) for theta.
 *   dL_du      device, d*nodes (vector-field layout), or NULL if L does not
 *              depend on u(T).
 *   dL_dtheta  device, nodes, or NULL if L does not depend on theta(T).
 * At least one must be given.  Requires a completed forward.
 * Errors: LB_EINVAL (both NULL), LB_ESTATE (no forward, or the context was
 * stepped since), LB_ECUDA.
 */
lb_status lb_adjoint_seed(lb_adj *a, const double *dL_du, const double *dL_dtheta);

/*
 * Run `nsteps` reverse steps (the remaining count is T minus those done).
 * Whole checkpoint segments replay a recorded graph; the results do not
 * depend on how the steps are split across calls.  LB_ESTATE if the
 * context's walls were changed (lb_set_boundary) since lb_adjoint_forward:
 * the checkpoints belong to the old geometry.
 */
lb_status lb_adjoint_step(lb_adj *a, int64_t nsteps);

/*
 * After T reverse steps: dL/dtheta0 (device, nodes) and, if requested at
 * creation, dL/dnu (host, 1 value; NULL to skip).  Synchronises the stream.
 * Errors: LB_ESTATE if the reverse pass is incomplete; LB_EINVAL if a
 * fixed-point adjoint field left |value| < 2^59 (not seen in practice: the
 * field grows by less than 1.3x over a reverse pass, against 8x of headroom).
 */
lb_status lb_adjoint_result(lb_adj *a, double *dL_dtheta0, double *dL_dnu);

/* Workspace facts: {T, C, checkpoints, reverse steps done, bytes held}. */
lb_status lb_adjoint_info(const lb_adj *a, double *info);

#ifdef __cplusplus
}
#endif

#endif /* LB_ADJOINT_H */
