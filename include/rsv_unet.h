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

#ifdef __cplusplus
}
#endif

#endif /* RSV_UNET_H */
