/*
 * rsv_unet.h - C ABI of the learned pressure stage of librsv.so.
 *
 * The paper's CPR preconditioner (Section "CPR", two-stage form) solves a
 * pressure system in its first stage with "any" AMG-type solver (Section
 * "AMG"); the learned stage replaces that solver by a 3-D convolutional
 * U-Net trained to imitate one multigrid V-cycle of the pressure system.
 * The network and its training run on the tensor cores (BF16 operands,
 * FP32 accumulation).  The conventions of rsv.h hold (status returns, void*
 * streams, device pointers on the current device).
 *
 * Volumes are channels-last: element (k, j, i, c) of an nx*ny*nz volume with
 * leading dimension ld sits at ((k*ny + j)*nx + i)*ld + c, so voxel
 * (k, j, i) is grid cell c = nx*ny*k + nx*j + i.  BF16 values are passed as
 * uint16_t bit patterns.  A 3x3x3 weight is w[co][t][ci] with tap
 * t = 9*(dz+1) + 3*(dy+1) + (dx+1); a 1x1x1 weight is w[co][ci].
 */
#ifndef RSV_UNET_H
#define RSV_UNET_H

#include "rsv.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ convolutions
 * These are the kernels of the network's layers, exposed for testing and for
 * callers that build their own networks.  Each call allocates its scratch on
 * the stream, checks the device error word and synchronises the stream.
 *
 * rsv_conv3d_fwd: y[v, n] = f(sum_t sum_c w[n][t][c] * x[v + off_t, c]) with zero
 * padding, the cross-correlation of one 3x3x3 (taps = 27) or 1x1x1 (taps = 1)
 * layer.  f adds bias[n] (bias may be NULL), applies max(., 0) when relu != 0,
 * and multiplies by (mask[v][n] > 0) when mask is not NULL (the ReLU mask of
 * the input gradient).  Result as BF16 into y (ld ldy, may be NULL) and/or
 * FP32 into y32 ([V][co], may be NULL).
 * Requirements (RSV_EINVAL otherwise): ci and co multiples of 32; ldx >= ci,
 * ldy >= co, ldmask >= co, all multiples of 8; every pointer 16-byte aligned.
 * Returns RSV_ETIMEOUT if a bounded device wait ran out, RSV_ENOTSUP if the
 * driver offers no tensor-map encoder. */
RSV_API rsv_status rsv_conv3d_fwd(void *stream, int nx, int ny, int nz, int taps, int ci, int co,
                                  const uint16_t *x, int ldx, const uint16_t *w, const float *bias, int relu,
                                  const uint16_t *mask, int ldmask, uint16_t *y, int ldy, float *y32);

/* rsv_conv3d_dgrad: gradient of sum(gy * conv(x, w)) with respect to x, for a
 * 3x3x3 layer: gx[v, c] = m(sum_t sum_n w[n][t][c] * gy[v - off_t, n]), where m
 * multiplies by (mask[v][c] > 0) when mask is not NULL.  gx as BF16 (ld ldgx)
 * and/or FP32 ([V][ci]).  Requirements as rsv_conv3d_fwd with the roles of ci
 * and co exchanged. */
RSV_API rsv_status rsv_conv3d_dgrad(void *stream, int nx, int ny, int nz, int ci, int co, const uint16_t *gy,
                                    int ldgy, const uint16_t *w, const uint16_t *mask, int ldmask, uint16_t *gx,
                                    int ldgx, float *gx32);

/* rsv_conv3d_wgrad: gradients of sum(gy * conv(x, w) + gy * bias): gw[n][t][c] =
 * sum_v gy[v, n] * x[v + off_t, c] (FP32, [co][taps][ci]) and gb[n] = sum_v gy[v, n]
 * (FP32, may be NULL).  Requirements: nx a multiple of 8, ci and co multiples
 * of 32, ldx >= ci, ldgy >= co. */
RSV_API rsv_status rsv_conv3d_wgrad(void *stream, int nx, int ny, int nz, int taps, int ci, int co,
                                    const uint16_t *x, int ldx, const uint16_t *gy, int ldgy, float *gw, float *gb);

/* ------------------------------------------------------------------ the network
 * Architecture (levels L, channels ch[l] = base * 2^l, l = 0..L-1):
 *   encoder level l: (l > 0: 2x2x2 average pooling of level l-1's output)
 *                    -> 3x3x3 conv + bias + ReLU -> 3x3x3 conv + bias + ReLU
 *   decoder level l < L-1: concatenate [nearest-upsampled output of level l+1,
 *                    encoder output of level l] -> two (3x3x3 conv + bias + ReLU)
 *   head: 1x1x1 conv to one channel plus bias, no activation.
 * Input channels: r_p / s with s = sqrt(mean(r_p^2)), and (ln k - mean) / std
 * over the grid (a channel whose scale is zero is fed as zeros).  The stage's
 * output is s * head.  Activations and conv weights are BF16, sums FP32.
 *
 * Parameters are one FP32 array: per layer its weight ([co][27][ci], the
 * head's [1][ch[0]]) then its bias [co], layers in the order enc1a, enc1b,
 * enc2a, ..., encLb, dec(L-1)a, dec(L-1)b, ..., dec1a, dec1b, head (enc1a has
 * ci = 2; dec(l)a has ci = ch[l] + ch[l-1] in 1-based level numbering).
 *
 * Training: rsv_unet_train_step runs the forward pass, the loss
 * mean((head - target / s)^2) over the voxels, the backward pass and one
 * Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr; lr <= 0
 * computes the gradient only).  The target is the pressure correction the
 * network should imitate (for example one multigrid V-cycle applied to r_p).
 */
typedef struct rsv_unet rsv_unet;

/* Network for an nx*ny*nz grid.  Requirements (RSV_EINVAL otherwise): 1 <= levels
 * <= 5; base in {32, 64, 96, 128} with base * 2^(levels-1) <= 512; nx, ny, nz
 * divisible by 2^(levels-1) and nx / 2^(levels-1) a multiple of 8.  Parameters
 * start at zero (set them with rsv_unet_set_params).  Device memory: about
 * 2.2 KB per fine-grid voxel at base 32 (activations kept for training). */
RSV_API rsv_status rsv_unet_create(void *stream, int nx, int ny, int nz, int base, int levels, rsv_unet **out);
RSV_API void rsv_unet_destroy(rsv_unet *u);
RSV_API rsv_status rsv_unet_num_params(const rsv_unet *u, int64_t *n);
/* Copy the FP32 parameter array in (host or device); resets the Adam moments and step count. */
RSV_API rsv_status rsv_unet_set_params(rsv_unet *u, const float *params, int on_device);
RSV_API rsv_status rsv_unet_get_params(const rsv_unet *u, float *params, int on_device);
/* Gradient of the loss of the last rsv_unet_train_step, same layout as the parameters. */
RSV_API rsv_status rsv_unet_get_grads(const rsv_unet *u, float *grads, int on_device);
/* corr = s * U(r_p / s, ln k): rp, lnk and corr are device float64 arrays of
 * nx*ny*nz values in cell order.  Synchronises the stream. */
RSV_API rsv_status rsv_unet_apply(rsv_unet *u, const double *rp, const double *lnk, double *corr);
/* One training step on one sample (device float64 arrays of nx*ny*nz values);
 * *loss (host, may be NULL) receives the loss before the update. */
RSV_API rsv_status rsv_unet_train_step(rsv_unet *u, const double *rp, const double *lnk, const double *target,
                                       float lr, double *loss);

/* n training steps in a row, sample i = (rp[i], lnk[i], target[i]) (host arrays of
 * device pointers to float64 [nx*ny*nz]), each followed by an Adam step with
 * learning rate lr > 0; losses (host, may be NULL) receives the n losses.  The
 * stream is synchronised once, at the end. */
RSV_API rsv_status rsv_unet_train_batch(rsv_unet *u, int n, const double *const *rp, const double *const *lnk,
                                        const double *const *target, float lr, double *losses);

/* Checkpoints of a network in training: its FP32 parameters, both Adam moment
 * arrays and the Adam step count, so that training resumes exactly where it
 * stopped.  The file is a magic line "RSVUNET1", one line of JSON (format,
 * version 1, nx, ny, nz, base, levels, nparam, adam_step, dtype "float32",
 * endian "little", sections ["params", "adam_m", "adam_v"]), then the three
 * float32 arrays of nparam values in that order.  rsv_unet_load requires a
 * network of the same grid, base and levels (RSV_EINVAL otherwise, or for a
 * malformed or truncated file) and leaves the network unchanged on error.
 * Both synchronise the network's stream.  The paper has no learned stage; this
 * is the save/load of its extension's trained state. */
RSV_API rsv_status rsv_unet_save(const rsv_unet *u, const char *path);
RSV_API rsv_status rsv_unet_load(rsv_unet *u, const char *path);

/* ------------------------------------------------------------------ use inside the solver
 * rsv_solver_set_learned: the network u (on the solver matrix's grid, one
 * system) becomes the pressure stage of RSV_PC_CPR_LEARNED; lnk is ln k of the
 * grid's cells (host or device float64, copied).  The solver does not own u:
 * keep it alive while the solver uses it.  With RSV_PC_CPR_LEARNED, every CPR
 * application runs the network on the restricted residual instead of the
 * V-cycle, until the solve falls back to the V-cycle for its remaining
 * iterations: when the network's output holds a NaN or Inf, or when the
 * implicit residual norm falls by less than the fraction stall_drop over
 * stall_window consecutive iterations (stall_window <= 0 selects 10% over 5;
 * at most 64).  Both decisions are taken on the device; rsv_solve_info
 * .fallback_iter reports where.  Requirements: FP64 precision and the FGMRES
 * solver (the network is a nonlinear preconditioner), else RSV_ENOTSUP at
 * rsv_precond_setup. */
RSV_API rsv_status rsv_solver_set_learned(rsv_solver *s, rsv_unet *u, const double *lnk, int on_device,
                                          int stall_window, double stall_drop);

/* rsv_solver_record_pressure: from now on, every FP64 CPR application
 * (RSV_PC_CPR) copies its restricted right-hand side r_p = Pi_r f (nb values)
 * into buf + k*nb for k = 0, 1, ... up to max_samples (device float64 array
 * [max_samples][nb]).  These are the inputs of the pressure stage that the
 * plain solver generates: the training samples of the network (their targets
 * come from rsv_cpr_vcycle).  buf = NULL stops recording.  The count restarts
 * at zero; rsv_solver_recorded returns it (synchronises). */
RSV_API rsv_status rsv_solver_record_pressure(rsv_solver *s, double *buf, int max_samples);
RSV_API rsv_status rsv_solver_recorded(rsv_solver *s, int *count);

#ifdef __cplusplus
}
#endif

#endif /* RSV_UNET_H */
