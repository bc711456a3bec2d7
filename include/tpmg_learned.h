/*
 * tpmg_learned.h -- C ABI of the learned form of the TPMG solver.
 *
 * A small network, trained on solves that the method itself produces, takes
 * two places in the preconditioned CG of tpmg.h:
 *
 *  - COARSE: the solve on the coarsest multigrid level of the V-cycle
 *    (Algorithm 1 applies nu_coarse line-relaxation sweeps there) is replaced
 *    by the network's prediction of the coarse solution followed by one
 *    block-Jacobi line relaxation from it;
 *  - WARM: the initial guess of CG is the network's prediction of the solution
 *    from the right-hand side, followed by one block-Jacobi line relaxation
 *    (eq. BlockJacobi: the V-cycle's smoother) on the finest level.  The
 *    column operator couples the levels about 10^6 times more strongly than
 *    the identity term, so a small vertically oscillating error of the
 *    network would dominate the residual; the relaxation solves each column
 *    exactly and leaves only the horizontally coupled part of the error.
 *
 * With a network inside it the preconditioner is no longer a fixed linear map,
 * so the solve runs flexible CG (Polak-Ribiere coefficient; Notay, SIAM J. Sci.
 * Comput. 22 (2000)), and plain TPMG-PCG stays both the judge of the network's
 * output and the fallback (see tpmg_solve_learned).
 *
 * The network is a per-column multilayer perceptron of four affine layers
 *     2 n_r -> h -> h -> h -> n_r,  ReLU after the first three,
 * weights used in bfloat16 (rounded from FP32 master copies), activations and
 * accumulation in FP32.  Its input for column T of a level holds the
 * right-hand side as point values (cell integral / cell volume |T| v_k) of the
 * column and the flux-weighted mean (weights g_e / sum g_e of Appendix A) over
 * the three edge neighbours, all divided by the root mean square s of the
 * point values over the level; its output is the column of u / s.
 *
 * Parameter layout (tpmg_net_n_params floats): W_1 [h][2 n_r] row-major, b_1 [h],
 * W_2 [h][h], b_2 [h], W_3 [h][h], b_3 [h], W_4 [n_r][h], b_4 [n_r].
 *
 * Conventions are those of tpmg.h: d_* device pointers (current device), h_*
 * host pointers, the caller owns its buffers, errors as tpmg_status.  A network
 * orders its work on the stream given to tpmg_net_create.
 */
#ifndef TPMG_LEARNED_H
#define TPMG_LEARNED_H

#include <stddef.h>

#include "tpmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpmg_net tpmg_net;

/* Allocates a network for columns of n_r cells with hidden width `hidden`
 * (1..1024), parameters and Adam state zero.  cuda_stream: cudaStream_t (NULL =
 * legacy default stream).  Errors: INVALID_ARG, OOM, CUDA. */
tpmg_status tpmg_net_create(int n_r, int hidden, void *cuda_stream, tpmg_net **out);

/* Number of parameters (floats) of the layout above; 0 for NULL. */
size_t tpmg_net_n_params(const tpmg_net *net);

/* Copies tpmg_net_n_params floats from h_params into the FP32 masters, rounds
 * the bfloat16 weights from them and clears the Adam state.  Synchronous. */
tpmg_status tpmg_net_set_params(tpmg_net *net, const float *h_params);

/* Copies the FP32 masters to h_params.  Synchronous. */
tpmg_status tpmg_net_get_params(tpmg_net *net, float *h_params);

/* d_y [rows][n_r] = network(d_x [rows][2 n_r]) (float32, row-major), rows in
 * 1..4194240.  Asynchronous.  Errors: INVALID_ARG, OOM (workspace), CUDA. */
tpmg_status tpmg_net_forward(tpmg_net *net, const float *d_x, long rows, float *d_y);

/* Gradient of the loss  sum_{r,k} (y_rk - t_rk)^2 / (rows n_r)  with respect to
 * the parameters, for the bfloat16 weights the passes use, into d_grad
 * (tpmg_net_n_params floats, parameter layout).  h_loss (nullable): the loss;
 * when given the call synchronises.  Errors as tpmg_net_forward. */
tpmg_status tpmg_net_gradients(tpmg_net *net, const float *d_x, const float *d_t, long rows, float *d_grad,
                               double *h_loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, learning
 * rate lr >= 0) on the minibatch (d_x, d_t) of tpmg_net_gradients, then the
 * bfloat16 weights are rounded again from the masters.  h_loss (nullable):
 * the loss before the step (synchronises).  Errors as tpmg_net_forward. */
tpmg_status tpmg_net_train_step(tpmg_net *net, const float *d_x, const float *d_t, long rows, float lr,
                                double *h_loss);

/* Message of the last failed call on net ("" if none). */
const char *tpmg_net_last_error(const tpmg_net *net);

/* Releases the network (after synchronising its stream).  NULL is ignored.  A
 * network must be detached from every context before it is destroyed. */
void tpmg_net_destroy(tpmg_net *net);

/* ---- data for training, from solves of the method ------------------------ */

/* Network inputs of `rows` columns of multigrid level `level` of ctx for the
 * field d_f (doubles, n_cells*n_r of that level, cell integrals): d_cells
 * (device ints, nullable = columns 0..rows-1) selects the columns, d_x
 * receives [rows][2 n_r] floats (rows * n_r < 2^31).  The scale s is taken over the whole level
 * field; h_scale (nullable) receives it (synchronises).  Asynchronous on the
 * context stream otherwise.  Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_net_features(tpmg_ctx *ctx, int level, const double *d_f, const int *d_cells, long rows, float *d_x,
                              double *h_scale);

/* Training targets d_t [rows][n_r] = u / s for the solution d_u on `level`,
 * with s the scale of the features of d_f.  Asynchronous.  Errors as above. */
tpmg_status tpmg_net_targets(tpmg_ctx *ctx, int level, const double *d_f, const double *d_u, const int *d_cells,
                             long rows, float *d_t);

/* Records the right-hand side that the coarsest level receives in every
 * V-cycle that ctx runs kernel by kernel (graphs 0), as doubles, one
 * n_cells(0)*n_r block per V-cycle, into d_buf until `capacity` blocks are
 * held.  d_buf NULL stops the recording.  Requires the mixed-precision form,
 * n_levels >= 2 and graphs 0.  Errors: INVALID_ARG. */
tpmg_status tpmg_record_coarse(tpmg_ctx *ctx, double *d_buf, int capacity);

/* Blocks recorded since the last tpmg_record_coarse call. */
tpmg_status tpmg_record_count(const tpmg_ctx *ctx, int *count);

/* d_u0 = the coarsest-level solution for the right-hand side d_f0 (doubles,
 * n_cells(0)*n_r) by `sweeps` (1..64) symmetric sweeps of the V-cycle's
 * coarsest-level line relaxation from zero -- the coarse solve of Algorithm 1
 * with nu_coarse = sweeps, on the same BF16 stencil in FP32.  Mixed-precision
 * form only.  Asynchronous.  Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_coarse_solve(tpmg_ctx *ctx, const double *d_f0, double *d_u0, int sweeps);

/* ---- the learned solve ---------------------------------------------------- */

enum { TPMG_NET_COARSE = 0, TPMG_NET_WARM = 1 };

/* Attaches net in `role` to ctx (NULL detaches).  The network's columns must
 * have ctx's n_r.  COARSE needs the mixed-precision form and n_levels >= 2.
 * Allocates the inference workspace on first use.  Errors: INVALID_ARG, OOM. */
tpmg_status tpmg_attach_net(tpmg_ctx *ctx, int role, tpmg_net *net);

/* z = B r: one V-cycle of the mixed-precision form (as tpmg_vcycle) in which the
 * attached COARSE network's prediction replaces the coarsest-level solve (the
 * preconditioner of tpmg_solve_learned).  Asynchronous.  Errors: INVALID_ARG
 * (also when no COARSE network is attached), CUDA. */
tpmg_status tpmg_vcycle_learned(tpmg_ctx *ctx, const double *d_r, double *d_z);

/* d_u = s network(features(d_f)) for every column of the level of `role`
 * (COARSE: level 0, WARM: the finest level; doubles of that level's size) with
 * the network attached in that role, evaluated as inside the solve but without
 * the line relaxation that follows there.  Inside the solve the network runs as
 * one fused tensor-core kernel when its hidden width is 64 and n_r is a
 * multiple of 8 (inputs and activations rounded to bfloat16, FP32
 * accumulation): on tcgen05 with FP32 accumulators in tensor memory when n_r
 * is a multiple of 16 up to 128 and params.net_tcgen05 is set (the default),
 * else with mma.sync; otherwise layer by layer with FP32 activations.
 * Asynchronous.  Errors: INVALID_ARG (also: no network in `role`), CUDA. */
tpmg_status tpmg_net_predict(tpmg_ctx *ctx, int role, const double *d_f, double *d_u);

/* *flag = 1 if, since tpmg_setup, a network kernel on the tcgen05 tensor cores
 * (params.net_tcgen05) gave up waiting for its matrix multiplies, else 0.  Such
 * a kernel writes NaN over the outputs it could not compute, so that the
 * judge of the warm start and the breakdown test of the solve reject them.
 * Not part of the paper: a health check of this implementation.  Waits for
 * the context's stream.  Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_net_fault(tpmg_ctx *ctx, int *flag);

/* Bits of *info of tpmg_solve_learned. */
enum { TPMG_LEARNED_WARM_USED = 1,      /* the network's initial guess was kept */
       TPMG_LEARNED_WARM_REJECTED = 2,  /* its residual was not below ||f||: restarted from u = 0 */
       TPMG_LEARNED_FALLBACK = 4 };     /* plain TPMG-PCG finished the solve */

/* Flexible CG for A u = f with the attached networks, stopping when
 * ||r_k|| <= rtol ||f|| (the accuracy of a solve from u = 0, whatever the
 * initial guess).  Initial guess: the WARM network's prediction and one
 * line relaxation if a WARM network is attached, else d_u on entry; it is
 * kept only if ||f - A u_0|| < ||f||
 * (judge), else u_0 = 0.  Preconditioner: the mixed-precision V-cycle, with
 * the COARSE network as its coarsest-level solve if one is attached.  The loop
 * runs on the device (one graph launch).  Fallback: if it has not converged in
 * max_iter iterations, or broke down, plain TPMG-PCG (tpmg_solve) continues from
 * its last iterate (from u = 0 after a breakdown) to the same ||f||-relative
 * tolerance with max_iter more iterations.
 * *iters = all iterations (network phase + fallback), *rel_resid = ||r|| / ||f||,
 * *info (nullable) = TPMG_LEARNED_* bits, *fallback_iters (nullable) = the
 * fallback's share, *kernel_launches (nullable) = kernels the solve executed.
 * Needs the mixed-precision form; max_iter in 1..4095.
 * Returns the final status (OK, NOT_CONVERGED, BREAKDOWN, INVALID_ARG, CUDA). */
tpmg_status tpmg_solve_learned(tpmg_ctx *ctx, const double *d_f, double *d_u, double rtol, int max_iter,
                               int *iters, double *rel_resid, int *info, int *fallback_iters,
                               long long *kernel_launches);

#ifdef __cplusplus
}
#endif

#endif /* TPMG_LEARNED_H */
