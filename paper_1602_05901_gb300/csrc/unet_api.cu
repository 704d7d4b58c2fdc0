// C entry points of the learned pressure stage (include/rsv_unet.h).
#include <cuda_bf16.h>

#include "../../include/rsv_unet.h"
#include "common.cuh"
#include "conv.cuh"

using namespace rsv;

namespace {

constexpr uint64_t kConvTimeoutNs = 2000000000ull;  // 2 s per bounded wait

// Device error word plus optional scratch, released on every path.
struct CallScratch {
    cudaStream_t st;
    int *err = nullptr;
    void *buf = nullptr;
    explicit CallScratch(cudaStream_t s) : st(s) {}
    ~CallScratch() {
        if (err) cudaFreeAsync(err, st);
        if (buf) cudaFreeAsync(buf, st);
    }
    rsv_status init(size_t bytes) {
        RSV_CUDA_TRY(cudaMallocAsync((void **)&err, sizeof(int), st));
        RSV_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        if (bytes) RSV_CUDA_TRY(cudaMallocAsync(&buf, bytes, st));
        return RSV_OK;
    }
    rsv_status finish() {
        int h = 0;
        RSV_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        RSV_CUDA_TRY(cudaStreamSynchronize(st));
        return h ? (rsv_status)h : RSV_OK;
    }
};

const __nv_bfloat16 *bf(const uint16_t *p) { return reinterpret_cast<const __nv_bfloat16 *>(p); }
__nv_bfloat16 *bf(uint16_t *p) { return reinterpret_cast<__nv_bfloat16 *>(p); }

}  // namespace

extern "C" rsv_status rsv_conv3d_fwd(void *stream, int nx, int ny, int nz, int taps, int ci, int co, const uint16_t *x,
                                     int ldx, const uint16_t *w, const float *bias, int relu, const uint16_t *mask,
                                     int ldmask, uint16_t *y, int ldy, float *y32) {
    cudaStream_t st = (cudaStream_t)stream;
    CallScratch cs(st);
    RSV_TRY(cs.init(0));
    RSV_TRY(conv_fwd(st, ConvVol{nx, ny, nz}, taps, ci, co, bf(x), ldx, bf(w), bias, relu, bf(mask), ldmask, bf(y),
                     ldy, y32, cs.err, kConvTimeoutNs));
    return cs.finish();
}

extern "C" rsv_status rsv_conv3d_dgrad(void *stream, int nx, int ny, int nz, int ci, int co, const uint16_t *gy,
                                       int ldgy, const uint16_t *w, const uint16_t *mask, int ldmask, uint16_t *gx,
                                       int ldgx, float *gx32) {
    if (ci <= 0 || co <= 0 || !w) return RSV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CallScratch cs(st);
    RSV_TRY(cs.init((size_t)ci * 27 * co * 2));
    __nv_bfloat16 *wt = (__nv_bfloat16 *)cs.buf;
    RSV_TRY(conv_flip(st, ci, co, bf(w), wt));
    RSV_TRY(conv_fwd(st, ConvVol{nx, ny, nz}, 27, co, ci, bf(gy), ldgy, wt, nullptr, 0, bf(mask), ldmask, bf(gx), ldgx,
                     gx32, cs.err, kConvTimeoutNs));
    return cs.finish();
}

extern "C" rsv_status rsv_conv3d_wgrad(void *stream, int nx, int ny, int nz, int taps, int ci, int co,
                                       const uint16_t *x, int ldx, const uint16_t *gy, int ldgy, float *gw,
                                       float *gb) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || (taps != 1 && taps != 27) || ci <= 0 || co <= 0 || ci % 32 || co % 32)
        return RSV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CallScratch cs(st);
    RSV_TRY(cs.init(conv_wgrad_scratch(ConvVol{nx, ny, nz}, taps, ci, co)));
    RSV_TRY(conv_wgrad(st, ConvVol{nx, ny, nz}, taps, ci, co, bf(x), ldx, bf(gy), ldgy, gw, gb, cs.buf, cs.err,
                       kConvTimeoutNs));
    return cs.finish();
}
