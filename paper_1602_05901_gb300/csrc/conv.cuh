// Launchers of the tensor-core convolutions (conv_tc.cu) and the U-Net glue kernels.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rsv {

struct ConvVol {
    int nx, ny, nz;
};

// y[v, n] = epilogue(sum_t sum_c w[n][t][c] x[v + off_t, c]) for n < co.
// x: [V][ldx] BF16 (channels 0..ci-1 used), w: [co][taps][ci] BF16; epilogue:
// + bias[n] (optional), ReLU (optional), times (mask[v][n] > 0) (optional);
// stored as BF16 into y[v][ldy] and/or as FP32 into y32[v][co].
rsv_status conv_fwd(cudaStream_t st, ConvVol vol, int taps, int ci, int co, const __nv_bfloat16 *x, int ldx,
                    const __nv_bfloat16 *w, const float *bias, int relu, const __nv_bfloat16 *mask, int ldm,
                    __nv_bfloat16 *y, int ldy, float *y32, int *err, uint64_t timeout_ns,
                    const int *gate = nullptr);

// Weights of the input gradient: wt[ci][t][co] = w[co][26 - t][ci].
rsv_status conv_flip(cudaStream_t st, int ci, int co, const __nv_bfloat16 *w, __nv_bfloat16 *wt);

// Scratch bytes needed by conv_wgrad for this shape.
size_t conv_wgrad_scratch(ConvVol vol, int taps, int ci, int co);

// gw[co][t][ci] = sum_v gy[v, co] x[v + off_t, ci] (FP32), gb[co] = sum_v gy[v, co] (optional).
rsv_status conv_wgrad(cudaStream_t st, ConvVol vol, int taps, int ci, int co, const __nv_bfloat16 *x, int ldx,
                      const __nv_bfloat16 *gy, int ldgy, float *gw, float *gb, void *scratch, int *err,
                      uint64_t timeout_ns);

}  // namespace rsv
