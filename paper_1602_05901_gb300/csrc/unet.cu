// The learned pressure stage: a 3-D U-Net, its training step and its use as
// the pressure solver of CPR.
//
// Network (levels L, channels ch[l] = base * 2^l):
//   encoder level l: [avg-pool 2x2x2 of level l-1's output]  -> conv3+ReLU -> conv3+ReLU
//   decoder level l < L-1: concat(nearest-upsample(level l+1's output), encoder output l)
//                          -> conv3+ReLU -> conv3+ReLU
//   head: 1x1x1 conv to one channel, no activation.
// Inputs: r_p / s with s = rms(r_p), and ln k standardised over the grid;
// the correction returned is s * output.
//
// Storage (all channels-last BF16 unless noted):
//   * the first conv reads an explicit im2col of the two input channels
//     (27 taps x 2 channels, padded to 64), so it runs as a 1x1x1 GEMM;
//   * encoder level l's second conv (l < L-1) writes straight into the
//     channels [ch[l+1], ch[l+1] + ch[l]) of the decoder's concatenation
//     buffer at level l, and the upsampling writes channels [0, ch[l+1]), so
//     no concatenation copy exists;
//   * parameters: one FP32 array, per layer the weight [co][taps][ci] then
//     the bias [co], in the order enc1a, enc1b, ..., encLb, dec(L-1)a,
//     dec(L-1)b, ..., dec1a, dec1b, head; a BF16 copy feeds the tensor cores.
// BF16 rounding happens exactly where a tensor is stored; every sum is FP32
// (or FP64 for the loss and the input statistics).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rsv_unet.h"
#include "common.cuh"
#include "conv.cuh"
#include "unet.cuh"

namespace rsv {
namespace {

constexpr int kMaxNetLevels = 5;
constexpr int kRedBlk = 296;
constexpr uint64_t kTimeoutNs = 2000000000ull;

__device__ __forceinline__ float bfv(__nv_bfloat16 h) { return __bfloat162float(h); }
__device__ __forceinline__ __nv_bfloat16 tobf(float f) { return __float2bfloat16_rn(f); }

// ------------------------------------------------------------------ deterministic FP64 sums
// mode 0: sum rp^2 and sum lnk; mode 1: sum (lnk - mu)^2 with mu = stats[1] / V.
__global__ void __launch_bounds__(256) stats_partial(const double *__restrict__ rp, const double *__restrict__ lnk,
                                                     int64_t n, int mode, const double *__restrict__ stats,
                                                     double *__restrict__ part, const int *gate) {
    if (gate && *gate) return;
    __shared__ double r0[256], r1[256];
    double a = 0.0, b = 0.0;
    const double mu = mode ? stats[1] / (double)n : 0.0;
    for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        if (mode == 0) {
            a += rp[i] * rp[i];
            b += lnk[i];
        } else {
            const double d = lnk[i] - mu;
            a += d * d;
        }
    }
    r0[threadIdx.x] = a;
    r1[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            r0[threadIdx.x] += r0[threadIdx.x + w];
            r1[threadIdx.x] += r1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = r0[0];
        part[2 * blockIdx.x + 1] = r1[0];
    }
}

// stats: [0] sum rp^2, [1] sum lnk, [2] sum (lnk-mu)^2, [3] s = rms(rp), [4] mu, [5] sd
__global__ void stats_final(const double *__restrict__ part, int nblk, int64_t n, int mode, double *stats,
                            const int *gate) {
    if (threadIdx.x != 0 || (gate && *gate)) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nblk; ++i) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    if (mode == 0) {
        stats[0] = a;
        stats[1] = b;
        stats[3] = sqrt(a / (double)n);
        stats[4] = b / (double)n;
    } else {
        stats[2] = a;
        stats[5] = sqrt(a / (double)n);
    }
}

// xs[v] = (bf16(rp[v] / s), bf16((lnk[v] - mu) / sd)): the two standardised input channels.
__global__ void __launch_bounds__(256) standardise_inputs(const double *__restrict__ rp, const double *__restrict__ lnk,
                                                          const double *__restrict__ stats, int64_t V,
                                                          __nv_bfloat162 *__restrict__ xs, const int *gate) {
    if (gate && *gate) return;
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= V) return;
    const double s = stats[3], mu = stats[4], sd = stats[5];
    const float c0 = s > 0.0 ? (float)(rp[v] / s) : 0.0f;
    const float c1 = sd > 0.0 ? (float)((lnk[v] - mu) / sd) : 0.0f;
    xs[v] = __floats2bfloat162_rn(c0, c1);
}

// in[v][2t + c] = xs[v + off_t].c (zero outside the grid) for t < 27; channels 54..63 zero.
// Thread (v, t), t in [0, 32): one 4-byte store each, coalesced.
__global__ void __launch_bounds__(256) im2col_inputs(const __nv_bfloat162 *__restrict__ xs, int nx, int ny, int nz,
                                                     __nv_bfloat162 *__restrict__ in, const int *gate) {
    if (gate && *gate) return;
    const int plane = nx * ny;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t V = (int64_t)plane * nz;
    if (gid >= V * 32) return;
    const int v = (int)(gid >> 5);
    const int t = (int)(gid & 31);
    __nv_bfloat162 val = __floats2bfloat162_rn(0.0f, 0.0f);
    if (t < 27) {
        const int z = v / plane, r = v - z * plane;
        const int y = r / nx, x = r - y * nx;
        const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
        if (xx >= 0 && xx < nx && yy >= 0 && yy < ny && zz >= 0 && zz < nz) val = xs[zz * plane + yy * nx + xx];
    }
    in[gid] = val;
}

// out[v'][c] = bf16(mean of the 8 children of v'), child values src[v][off + c] (ld lds).
__global__ void __launch_bounds__(256) avgpool_bf16(const __nv_bfloat16 *__restrict__ src, int lds, int C, int nx,
                                                    int ny, int nz, __nv_bfloat16 *__restrict__ dst,
                                                    const int *gate) {
    if (gate && *gate) return;
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int64_t total = (int64_t)cx * cy * cz * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t vc = i / C;
        const int x = (int)(vc % cx), y = (int)((vc / cx) % cy), z = (int)(vc / ((int64_t)cx * cy));
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t u = ((int64_t)(2 * z + (k >> 2)) * ny + (2 * y + ((k >> 1) & 1))) * nx + 2 * x + (k & 1);
            s += bfv(src[u * lds + c]);
        }
        dst[i] = tobf(s * 0.125f);
    }
}

// dst[v][c] = src[parent(v)][c] for c < C (fine volume nx*ny*nz, dst ld ldd), 8 channels per thread.
__global__ void __launch_bounds__(256) upsample_bf16(const __nv_bfloat16 *__restrict__ src, int C, int nx, int ny,
                                                     int nz, __nv_bfloat16 *__restrict__ dst, int ldd,
                                                     const int *gate) {
    if (gate && *gate) return;
    const int c8 = C / 8;
    const int64_t total = (int64_t)nx * ny * nz * c8;
    const int cx = nx / 2, cy = ny / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(i % c8);
        const int64_t v = i / c8;
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
        const int64_t p = ((int64_t)(z / 2) * cy + y / 2) * cx + x / 2;
        ((uint4 *)(dst + v * ldd))[q] = ((const uint4 *)(src + p * C))[q];
    }
}

// g[v'][c] = bf16( sum over the 8 children of gcat[child][c] , times (act[v'][c] > 0) ), coarse voxel v'.
__global__ void __launch_bounds__(256) upsample_bwd_mask(const __nv_bfloat16 *__restrict__ gcat, int ldg, int C,
                                                         int nx, int ny, int nz, const __nv_bfloat16 *__restrict__ act,
                                                         int lda, __nv_bfloat16 *__restrict__ g) {
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int64_t total = (int64_t)cx * cy * cz * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t vc = i / C;
        const int x = (int)(vc % cx), y = (int)((vc / cx) % cy), z = (int)(vc / ((int64_t)cx * cy));
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t u = ((int64_t)(2 * z + (k >> 2)) * ny + (2 * y + ((k >> 1) & 1))) * nx + 2 * x + (k & 1);
            s += bfv(gcat[u * ldg + c]);
        }
        g[i] = tobf(bfv(act[vc * lda + c]) > 0.0f ? s : 0.0f);
    }
}

// g[v][c] = bf16( (skip[v][c] + gp[parent(v)][c] / 8) * (act[v][c] > 0) ), fine voxel v.
__global__ void __launch_bounds__(256) combine_skip_pool(const __nv_bfloat16 *__restrict__ skip, int lds,
                                                         const __nv_bfloat16 *__restrict__ gp, int C, int nx, int ny,
                                                         int nz, const __nv_bfloat16 *__restrict__ act, int lda,
                                                         __nv_bfloat16 *__restrict__ g) {
    const int64_t total = (int64_t)nx * ny * nz * C;
    const int cx = nx / 2, cy = ny / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t v = i / C;
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
        const int64_t p = ((int64_t)(z / 2) * cy + y / 2) * cx + x / 2;
        const float s = bfv(skip[v * lds + c]) + bfv(gp[p * C + c]) * 0.125f;
        g[i] = tobf(bfv(act[v * lda + c]) > 0.0f ? s : 0.0f);
    }
}

// out[v] = sum_c top[v][c] wh[c] + bh (FP32); corr[v] = s * out[v] (optional).
__global__ void __launch_bounds__(256) head_fwd(const __nv_bfloat16 *__restrict__ top, int C, int64_t V,
                                                const float *__restrict__ wh, const double *__restrict__ stats,
                                                float *__restrict__ out, double *__restrict__ corr, const int *gate) {
    if (gate && *gate) return;
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= V) return;
    float acc = 0.0f;
    for (int c = 0; c < C; ++c) acc = fmaf(bfv(top[v * C + c]), wh[c], acc);
    acc += wh[C];
    out[v] = acc;
    if (corr) corr[v] = stats[3] > 0.0 ? stats[3] * (double)acc : 0.0;
}

// Loss and the head's gradients.  d = out - target / s; loss = mean d^2;
// gout = 2 d / V; G[v][c] = bf16(gout wh[c] (top > 0)).  Each CTA owns a
// contiguous chunk of voxels and each warp 32 consecutive voxels at a time:
// lane l first forms d and gout of voxel l (the FP64 part, once per voxel),
// then the warp walks the 32 voxels with lane l on channels l, l + 32, ...
// (C <= 128), so each voxel's row is read and written coalesced.  Per-CTA
// sums of gout * top[v][c] (c < C), of gout (slot C) and of d^2 (slot C + 1)
// go to part[blockIdx.x][C + 2], warps added in order; head_final adds the
// CTAs in order.
__global__ void __launch_bounds__(256) head_bwd(const __nv_bfloat16 *__restrict__ top, int C, int64_t V,
                                                const float *__restrict__ wh, const float *__restrict__ out,
                                                const double *__restrict__ tgt, const double *__restrict__ stats,
                                                __nv_bfloat16 *__restrict__ G, double *__restrict__ part) {
    __shared__ double red[8][130];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t len = (V + gridDim.x - 1) / gridDim.x;
    const int64_t v0 = blockIdx.x * len, v1 = min(V, v0 + len);
    const double s = stats[3];
    const double inv_s = s > 0.0 ? 1.0 / s : 0.0, two_over_v = 2.0 / (double)V;
    float w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = lane + 32 * q < C ? wh[lane + 32 * q] : 0.0f;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    double gsum = 0.0, dsum = 0.0;
    for (int64_t b = v0 + 32 * warp; b < v1; b += 256) {
        const int64_t vl = b + lane;
        float g = 0.0f;
        if (vl < v1) {
            const double d = (double)out[vl] - tgt[vl] * inv_s;
            g = (float)(d * two_over_v);
            gsum += g;
            dsum += d * d;
        }
        const int nv = v1 - b < 32 ? (int)(v1 - b) : 32;
        for (int j = 0; j < nv; ++j) {
            const float gj = __shfl_sync(0xffffffffu, g, j);
            const int64_t v = b + j;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                if (c < C) {
                    const float a = bfv(top[v * C + c]);
                    G[v * C + c] = tobf(a > 0.0f ? gj * w[q] : 0.0f);
                    acc[q] = fmaf(gj, a, acc[q]);
                }
            }
        }
    }
    // warp sums of the per-voxel scalars, then per-CTA sums over the warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gsum += __shfl_down_sync(0xffffffffu, gsum, o);
        dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (lane + 32 * q < C) red[warp][lane + 32 * q] = acc[q];
    if (lane == 0) {
        red[warp][C] = gsum;
        red[warp][C + 1] = dsum;
    }
    __syncthreads();
    if (threadIdx.x < C + 2) {
        double t = 0.0;
        for (int wv = 0; wv < 8; ++wv) t += red[wv][threadIdx.x];
        part[(int64_t)blockIdx.x * (C + 2) + threadIdx.x] = t;
    }
}

// Head gradients into the flat gradient array, and the loss: grad[gw + c], grad[gw + C], loss.
__global__ void head_final(const double *__restrict__ part, int nblk, int C, int64_t V, float *__restrict__ grad,
                           double *__restrict__ loss) {
    const int k = threadIdx.x;
    if (k >= C + 2) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * (C + 2) + k];
    if (k <= C)
        grad[k] = (float)s;
    else
        *loss = s / (double)V;
}

// One Adam step on every parameter, then the BF16 copy.  c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t).
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16 *__restrict__ pw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        pw[i] = tobf(pi);
    }
}

__global__ void to_bf16(const float *__restrict__ p, int64_t n, __nv_bfloat16 *__restrict__ pw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pw[i] = tobf(p[i]);
}

// im2col weights of the first layer: w1c[co][k] = w[co][k] for k < 54 (k = 2t + c), zero for k in [54, 64).
__global__ void pack_first(const float *__restrict__ w, int co, __nv_bfloat16 *__restrict__ w1c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= co * 64) return;
    const int o = i / 64, k = i % 64;
    w1c[i] = tobf(k < 54 ? w[o * 54 + k] : 0.0f);
}
__global__ void unpack_first_grad(const float *__restrict__ g1c, int co, float *__restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= co * 54) return;
    g[i] = g1c[(i / 54) * 64 + i % 54];
}

int blocks_for(int64_t n, int per = 256, int cap = 8192) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, cap));
}

}  // namespace

struct Layer {
    int co, ci, taps;
    int64_t woff, boff;  // offsets in the flat parameter array
};

}  // namespace rsv

using namespace rsv;

struct rsv_unet {
    cudaStream_t st = nullptr;
    int nx = 0, ny = 0, nz = 0, base = 0, L = 0;
    int ch[kMaxNetLevels] = {};
    ConvVol vol[kMaxNetLevels] = {};
    int64_t V[kMaxNetLevels] = {};
    int catC[kMaxNetLevels] = {};
    std::vector<Layer> layers;  // 2L (encoder) + 2(L-1) (decoder) + head
    int64_t nparam = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pw = nullptr, *w1c = nullptr, *wflip = nullptr;
    float *g1c = nullptr;
    __nv_bfloat16 *in = nullptr, *ebL = nullptr;
    __nv_bfloat162 *xs = nullptr;  // the two standardised input channels per voxel
    __nv_bfloat16 *ea[kMaxNetLevels] = {}, *cat[kMaxNetLevels] = {}, *da[kMaxNetLevels] = {}, *db[kMaxNetLevels] = {},
                  *pool[kMaxNetLevels] = {};
    __nv_bfloat16 *gA[kMaxNetLevels] = {}, *gB[kMaxNetLevels] = {}, *gcat[kMaxNetLevels] = {}, *gp[kMaxNetLevels] = {};
    float *out = nullptr;
    double *stats = nullptr, *part = nullptr, *loss = nullptr;
    void *wscratch = nullptr;
    int *err = nullptr;
    int adam_t = 0;
    const int *gate = nullptr;  // forward kernels skip when *gate != 0 (solver use)
    bool acts_valid = false;  // activations of the last forward pass are kept (train step needs them)
    std::vector<void *> allocs;

    // layer indices
    int enc_a(int l) const { return 2 * l; }
    int enc_b(int l) const { return 2 * l + 1; }
    int dec_a(int l) const { return 2 * L + 2 * (L - 2 - l); }
    int dec_b(int l) const { return dec_a(l) + 1; }
    int head() const { return (int)layers.size() - 1; }
    const __nv_bfloat16 *W(int i) const { return pw + layers[i].woff; }
    const float *B(int i) const { return p + layers[i].boff; }
    // output of encoder level l's second conv (pointer, leading dimension)
    __nv_bfloat16 *eb(int l) const { return l == L - 1 ? ebL : cat[l] + ch[l + 1]; }
    int ldeb(int l) const { return l == L - 1 ? ch[l] : catC[l]; }
    __nv_bfloat16 *top() const { return L > 1 ? db[0] : ebL; }

    ~rsv_unet() {
        for (void *q : allocs) cudaFree(q);
    }
    template <typename T>
    rsv_status alloc(T **ptr, size_t count) {
        void *q = nullptr;
        RSV_CUDA_TRY(cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16)));
        allocs.push_back(q);
        *ptr = (T *)q;
        return RSV_OK;
    }
};

namespace rsv {
namespace {

rsv_status unet_alloc(rsv_unet *u) {
    const int L = u->L;
    // parameters
    int64_t off = 0;
    for (int l = 0; l < L; ++l) {
        const int ci_a = l == 0 ? 2 : u->ch[l - 1];
        u->layers.push_back({u->ch[l], ci_a, 27, off, off + (int64_t)u->ch[l] * 27 * ci_a});
        off = u->layers.back().boff + u->ch[l];
        u->layers.push_back({u->ch[l], u->ch[l], 27, off, off + (int64_t)u->ch[l] * 27 * u->ch[l]});
        off = u->layers.back().boff + u->ch[l];
    }
    for (int l = L - 2; l >= 0; --l) {
        u->layers.push_back({u->ch[l], u->catC[l], 27, off, off + (int64_t)u->ch[l] * 27 * u->catC[l]});
        off = u->layers.back().boff + u->ch[l];
        u->layers.push_back({u->ch[l], u->ch[l], 27, off, off + (int64_t)u->ch[l] * 27 * u->ch[l]});
        off = u->layers.back().boff + u->ch[l];
    }
    u->layers.push_back({1, u->ch[0], 1, off, off + u->ch[0]});
    off += u->ch[0] + 1;
    u->nparam = off;
    const int64_t np8 = (u->nparam + 7) / 8 * 8;
    RSV_TRY(u->alloc(&u->p, np8));
    RSV_TRY(u->alloc(&u->g, np8));
    RSV_TRY(u->alloc(&u->m, np8));
    RSV_TRY(u->alloc(&u->v, np8));
    RSV_TRY(u->alloc(&u->pw, np8));
    RSV_TRY(u->alloc(&u->w1c, (size_t)u->ch[0] * 64));
    RSV_TRY(u->alloc(&u->g1c, (size_t)u->ch[0] * 64));
    size_t flip = 0, wscr = 0;
    for (size_t i = 0; i + 1 < u->layers.size(); ++i)
        flip = std::max(flip, (size_t)u->layers[i].co * 27 * u->layers[i].ci);
    RSV_TRY(u->alloc(&u->wflip, flip));
    // activations and gradients
    RSV_TRY(u->alloc(&u->in, (size_t)u->V[0] * 64));
    RSV_TRY(u->alloc(&u->xs, (size_t)u->V[0]));
    for (int l = 0; l < L; ++l) {
        const size_t V = (size_t)u->V[l], c = (size_t)u->ch[l];
        RSV_TRY(u->alloc(&u->ea[l], V * c));
        RSV_TRY(u->alloc(&u->gA[l], V * std::max<size_t>(c, l > 0 ? (size_t)u->ch[l - 1] : c)));
        RSV_TRY(u->alloc(&u->gB[l], V * c));
        if (l > 0) {
            RSV_TRY(u->alloc(&u->pool[l], V * u->ch[l - 1]));
            RSV_TRY(u->alloc(&u->gp[l], V * u->ch[l - 1]));
        }
        if (l < L - 1) {
            RSV_TRY(u->alloc(&u->cat[l], V * u->catC[l]));
            RSV_TRY(u->alloc(&u->gcat[l], V * u->catC[l]));
            RSV_TRY(u->alloc(&u->da[l], V * c));
            RSV_TRY(u->alloc(&u->db[l], V * c));
        }
    }
    RSV_TRY(u->alloc(&u->ebL, (size_t)u->V[L - 1] * u->ch[L - 1]));
    for (size_t i = 0; i + 1 < u->layers.size(); ++i) {
        const Layer &ly = u->layers[i];
        int l = 0;  // level of layer i
        if ((int)i < 2 * L)
            l = (int)i / 2;
        else
            l = L - 2 - ((int)i - 2 * L) / 2;
        wscr = std::max(wscr, conv_wgrad_scratch(u->vol[l], i == 0 ? 1 : 27, i == 0 ? 64 : ly.ci, ly.co));
    }
    RSV_TRY(u->alloc((char **)&u->wscratch, wscr));
    RSV_TRY(u->alloc(&u->out, (size_t)u->V[0]));
    RSV_TRY(u->alloc(&u->stats, 16));
    RSV_TRY(u->alloc(&u->part, (size_t)kRedBlk * (u->ch[0] + 2)));
    RSV_TRY(u->alloc(&u->loss, 1));
    RSV_TRY(u->alloc(&u->err, 1));
    RSV_CUDA_TRY(cudaMemsetAsync(u->err, 0, sizeof(int), u->st));
    return RSV_OK;
}

rsv_status conv(rsv_unet *u, int l, int layer, const __nv_bfloat16 *x, int ldx, __nv_bfloat16 *y, int ldy) {
    const Layer &ly = u->layers[layer];
    return conv_fwd(u->st, u->vol[l], 27, ly.ci, ly.co, x, ldx, u->W(layer), u->B(layer), 1, nullptr, 0, y, ldy,
                    nullptr, u->err, kTimeoutNs, u->gate);
}

// Forward pass; keeps every activation for the backward pass.  corr (optional) = s * output.
rsv_status forward(rsv_unet *u, const double *rp, const double *lnk, double *corr) {
    cudaStream_t st = u->st;
    const int L = u->L;
    const int64_t V0 = u->V[0];
    const int *gate = u->gate;
    stats_partial<<<kRedBlk, 256, 0, st>>>(rp, lnk, V0, 0, u->stats, u->part, gate);
    stats_final<<<1, 32, 0, st>>>(u->part, kRedBlk, V0, 0, u->stats, gate);
    stats_partial<<<kRedBlk, 256, 0, st>>>(rp, lnk, V0, 1, u->stats, u->part, gate);
    stats_final<<<1, 32, 0, st>>>(u->part, kRedBlk, V0, 1, u->stats, gate);
    standardise_inputs<<<blocks_for(V0, 256, 1 << 30), 256, 0, st>>>(rp, lnk, u->stats, V0, u->xs, gate);
    im2col_inputs<<<blocks_for(V0 * 32, 256, 1 << 30), 256, 0, st>>>(u->xs, u->nx, u->ny, u->nz,
                                                                     (__nv_bfloat162 *)u->in, gate);
    RSV_CUDA_TRY(cudaGetLastError());
    count_launches(6);
    // first layer: 1x1x1 GEMM over the im2col channels
    RSV_TRY(conv_fwd(st, u->vol[0], 1, 64, u->ch[0], u->in, 64, u->w1c, u->B(0), 1, nullptr, 0, u->ea[0], u->ch[0],
                     nullptr, u->err, kTimeoutNs, gate));
    for (int l = 0; l < L; ++l) {
        if (l > 0) {
            const ConvVol &f = u->vol[l - 1];
            avgpool_bf16<<<blocks_for(u->V[l] * u->ch[l - 1]), 256, 0, st>>>(u->eb(l - 1), u->ldeb(l - 1), u->ch[l - 1],
                                                                              f.nx, f.ny, f.nz, u->pool[l], gate);
            RSV_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            RSV_TRY(conv(u, l, u->enc_a(l), u->pool[l], u->ch[l - 1], u->ea[l], u->ch[l]));
        }
        RSV_TRY(conv(u, l, u->enc_b(l), u->ea[l], u->ch[l], u->eb(l), u->ldeb(l)));
    }
    for (int l = L - 2; l >= 0; --l) {
        const __nv_bfloat16 *src = l == L - 2 ? u->ebL : u->db[l + 1];
        const ConvVol &f = u->vol[l];
        upsample_bf16<<<blocks_for(u->V[l] * u->ch[l + 1] / 8), 256, 0, st>>>(src, u->ch[l + 1], f.nx, f.ny, f.nz,
                                                                              u->cat[l], u->catC[l], gate);
        RSV_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        RSV_TRY(conv(u, l, u->dec_a(l), u->cat[l], u->catC[l], u->da[l], u->ch[l]));
        RSV_TRY(conv(u, l, u->dec_b(l), u->da[l], u->ch[l], u->db[l], u->ch[l]));
    }
    head_fwd<<<blocks_for(V0, 256, 1 << 30), 256, 0, st>>>(u->top(), u->ch[0], V0, u->p + u->layers[u->head()].woff,
                                                           u->stats, u->out, corr, gate);
    RSV_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    u->acts_valid = true;
    return RSV_OK;
}

rsv_status conv_back(rsv_unet *u, int l, int layer, const __nv_bfloat16 *x, int ldx, const __nv_bfloat16 *gy,
                     const __nv_bfloat16 *mask, int ldm, __nv_bfloat16 *gx, int ldgx) {
    const Layer &ly = u->layers[layer];
    cudaStream_t st = u->st;
    RSV_TRY(conv_wgrad(st, u->vol[l], 27, ly.ci, ly.co, x, ldx, gy, ly.co, u->g + ly.woff, u->g + ly.boff,
                       u->wscratch, u->err, kTimeoutNs));
    if (!gx) return RSV_OK;
    RSV_TRY(conv_flip(st, ly.ci, ly.co, u->W(layer), u->wflip));
    return conv_fwd(st, u->vol[l], 27, ly.co, ly.ci, gy, ly.co, u->wflip, nullptr, 0, mask, ldm, gx, ldgx, nullptr,
                    u->err, kTimeoutNs);
}

// Backward pass of the loss mean((out - target/s)^2) after forward(); gradients into u->g.
rsv_status backward(rsv_unet *u, const double *target) {
    cudaStream_t st = u->st;
    const int L = u->L;
    const int64_t V0 = u->V[0];
    const int C0 = u->ch[0];
    const Layer &hd = u->layers[u->head()];
    head_bwd<<<kRedBlk, 256, 0, st>>>(u->top(), C0, V0, u->p + hd.woff, u->out, target, u->stats, u->gB[0], u->part);
    head_final<<<1, (C0 + 2 + 31) / 32 * 32, 0, st>>>(u->part, kRedBlk, C0, V0, u->g + hd.woff, u->loss);
    RSV_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    // decoder, top level first
    for (int l = 0; l < L - 1; ++l) {
        RSV_TRY(conv_back(u, l, u->dec_b(l), u->da[l], u->ch[l], u->gB[l], u->da[l], u->ch[l], u->gA[l], u->ch[l]));
        RSV_TRY(conv_back(u, l, u->dec_a(l), u->cat[l], u->catC[l], u->gA[l], nullptr, 0, u->gcat[l], u->catC[l]));
        const __nv_bfloat16 *below = l + 1 == L - 1 ? u->ebL : u->db[l + 1];
        const ConvVol &f = u->vol[l];
        upsample_bwd_mask<<<blocks_for(u->V[l + 1] * u->ch[l + 1]), 256, 0, st>>>(
            u->gcat[l], u->catC[l], u->ch[l + 1], f.nx, f.ny, f.nz, below, u->ch[l + 1], u->gB[l + 1]);
        RSV_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    }
    // encoder, deepest level first
    for (int l = L - 1; l >= 0; --l) {
        RSV_TRY(conv_back(u, l, u->enc_b(l), u->ea[l], u->ch[l], u->gB[l], u->ea[l], u->ch[l], u->gA[l], u->ch[l]));
        if (l == 0) {
            RSV_TRY(conv_wgrad(st, u->vol[0], 1, 64, C0, u->in, 64, u->gA[0], C0, u->g1c, u->g + u->layers[0].boff,
                               u->wscratch, u->err, kTimeoutNs));
            unpack_first_grad<<<(C0 * 54 + 255) / 256, 256, 0, st>>>(u->g1c, C0, u->g + u->layers[0].woff);
            RSV_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            break;
        }
        RSV_TRY(conv_back(u, l, u->enc_a(l), u->pool[l], u->ch[l - 1], u->gA[l], nullptr, 0, u->gp[l], u->ch[l - 1]));
        const ConvVol &f = u->vol[l - 1];
        combine_skip_pool<<<blocks_for(u->V[l - 1] * u->ch[l - 1]), 256, 0, st>>>(
            u->gcat[l - 1] + u->ch[l], u->catC[l - 1], u->gp[l], u->ch[l - 1], f.nx, f.ny, f.nz, u->eb(l - 1),
            u->ldeb(l - 1), u->gB[l - 1]);
        RSV_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    }
    return RSV_OK;
}

rsv_status refresh_bf16(rsv_unet *u) {
    to_bf16<<<blocks_for(u->nparam), 256, 0, u->st>>>(u->p, u->nparam, u->pw);
    pack_first<<<(u->ch[0] * 64 + 255) / 256, 256, 0, u->st>>>(u->p + u->layers[0].woff, u->ch[0], u->w1c);
    RSV_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return RSV_OK;
}

rsv_status check_err(rsv_unet *u) {
    int h = 0;
    RSV_CUDA_TRY(cudaMemcpyAsync(&h, u->err, sizeof(int), cudaMemcpyDeviceToHost, u->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(u->st));
    if (h) {
        cudaMemsetAsync(u->err, 0, sizeof(int), u->st);
        return (rsv_status)h;
    }
    return RSV_OK;
}

}  // namespace

rsv_status unet_apply_device(rsv_unet *u, cudaStream_t st, const double *rp, const double *lnk, double *corr,
                             const int *gate) {
    cudaStream_t saved = u->st;
    u->st = st;
    u->gate = gate;
    rsv_status s = forward(u, rp, lnk, corr);
    u->st = saved;
    u->gate = nullptr;
    return s;
}

void unet_dims(const rsv_unet *u, int *nx, int *ny, int *nz) {
    *nx = u->nx;
    *ny = u->ny;
    *nz = u->nz;
}

int unet_error(rsv_unet *u, cudaStream_t st) {
    int h = 0;
    if (cudaMemcpyAsync(&h, u->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RSV_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSV_ECUDA;
    return h;
}

}  // namespace rsv

// ------------------------------------------------------------------ C entry points
extern "C" rsv_status rsv_unet_create(void *stream, int nx, int ny, int nz, int base, int levels, rsv_unet **out) {
    if (!out || levels < 1 || levels > kMaxNetLevels || base < 32 || base > 128 || base % 32 || nx <= 0 || ny <= 0 ||
        nz <= 0)
        return RSV_EINVAL;
    const int q = 1 << (levels - 1);
    if (nx % q || ny % q || nz % q || (nx / q) % 8 || (int64_t)nx * ny * nz > (1ll << 31) / 64 ||
        (int64_t)base << (levels - 1) > 512)
        return RSV_EINVAL;
    rsv_unet *u = new (std::nothrow) rsv_unet();
    if (!u) return RSV_ENOMEM;
    u->st = (cudaStream_t)stream;
    u->nx = nx;
    u->ny = ny;
    u->nz = nz;
    u->base = base;
    u->L = levels;
    for (int l = 0; l < levels; ++l) {
        u->ch[l] = base << l;
        u->vol[l] = ConvVol{nx >> l, ny >> l, nz >> l};
        u->V[l] = (int64_t)(nx >> l) * (ny >> l) * (nz >> l);
        u->catC[l] = l + 1 < levels ? (base << (l + 1)) + (base << l) : 0;
    }
    rsv_status s = unet_alloc(u);
    if (s == RSV_OK) {
        cudaError_t e = cudaMemsetAsync(u->p, 0, sizeof(float) * u->nparam, u->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(u->m, 0, sizeof(float) * u->nparam, u->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(u->v, 0, sizeof(float) * u->nparam, u->st);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            s = RSV_ECUDA;
        }
    }
    if (s == RSV_OK) s = refresh_bf16(u);
    if (s != RSV_OK) {
        delete u;
        return s;
    }
    *out = u;
    return RSV_OK;
}

extern "C" void rsv_unet_destroy(rsv_unet *u) {
    if (!u) return;
    cudaStreamSynchronize(u->st);
    delete u;
}

extern "C" rsv_status rsv_unet_num_params(const rsv_unet *u, int64_t *n) {
    if (!u || !n) return RSV_EINVAL;
    *n = u->nparam;
    return RSV_OK;
}

extern "C" rsv_status rsv_unet_set_params(rsv_unet *u, const float *params, int on_device) {
    if (!u || !params) return RSV_EINVAL;
    RSV_CUDA_TRY(cudaMemcpyAsync(u->p, params, sizeof(float) * u->nparam,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, u->st));
    RSV_CUDA_TRY(cudaMemsetAsync(u->m, 0, sizeof(float) * u->nparam, u->st));
    RSV_CUDA_TRY(cudaMemsetAsync(u->v, 0, sizeof(float) * u->nparam, u->st));
    u->adam_t = 0;
    RSV_TRY(refresh_bf16(u));
    RSV_CUDA_TRY(cudaStreamSynchronize(u->st));
    return RSV_OK;
}

static rsv_status copy_out(const rsv_unet *u, const float *src, float *dst, int on_device) {
    if (!u || !dst) return RSV_EINVAL;
    RSV_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(float) * u->nparam,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(u->st));
    return RSV_OK;
}

extern "C" rsv_status rsv_unet_get_params(const rsv_unet *u, float *params, int on_device) {
    return u ? copy_out(u, u->p, params, on_device) : RSV_EINVAL;
}

extern "C" rsv_status rsv_unet_get_grads(const rsv_unet *u, float *grads, int on_device) {
    return u ? copy_out(u, u->g, grads, on_device) : RSV_EINVAL;
}

// ---- checkpoints: a text header line (JSON) then params, Adam m, Adam v as little-endian float32
namespace {

constexpr char kCkptMagic[] = "RSVUNET1\n";

bool read_json_int(const std::string &h, const char *key, long long *out) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = h.find(k);
    if (at == std::string::npos) return false;
    return std::sscanf(h.c_str() + at + k.size(), " %lld", out) == 1;
}

}  // namespace

extern "C" rsv_status rsv_unet_save(const rsv_unet *u, const char *path) {
    if (!u || !path) return RSV_EINVAL;
    std::vector<float> buf;
    try {
        buf.resize(3 * (size_t)u->nparam);
    } catch (...) {
        return RSV_ENOMEM;
    }
    const float *src[3] = {u->p, u->m, u->v};
    for (int q = 0; q < 3; ++q)
        RSV_CUDA_TRY(cudaMemcpyAsync(buf.data() + q * (size_t)u->nparam, src[q], sizeof(float) * u->nparam,
                                     cudaMemcpyDeviceToHost, u->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(u->st));
    char head[512];
    const int len = std::snprintf(head, sizeof head,
                                  "{\"format\":\"rsv_unet\",\"version\":1,\"nx\":%d,\"ny\":%d,\"nz\":%d,"
                                  "\"base\":%d,\"levels\":%d,\"nparam\":%lld,\"adam_step\":%d,"
                                  "\"dtype\":\"float32\",\"endian\":\"little\","
                                  "\"sections\":[\"params\",\"adam_m\",\"adam_v\"]}\n",
                                  u->nx, u->ny, u->nz, u->base, u->L, (long long)u->nparam, u->adam_t);
    if (len <= 0 || len >= (int)sizeof head) return RSV_EINVAL;
    FILE *f = std::fopen(path, "wb");
    if (!f) return RSV_EINVAL;
    bool ok = std::fwrite(kCkptMagic, 1, sizeof kCkptMagic - 1, f) == sizeof kCkptMagic - 1 &&
              std::fwrite(head, 1, (size_t)len, f) == (size_t)len &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? RSV_OK : RSV_EINVAL;
}

extern "C" rsv_status rsv_unet_load(rsv_unet *u, const char *path) {
    if (!u || !path) return RSV_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f) return RSV_EINVAL;
    char magic[sizeof kCkptMagic - 1];
    char line[512];
    rsv_status st = RSV_OK;
    std::vector<float> buf;
    if (std::fread(magic, 1, sizeof magic, f) != sizeof magic || std::memcmp(magic, kCkptMagic, sizeof magic) ||
        !std::fgets(line, sizeof line, f))
        st = RSV_EINVAL;
    long long nx = 0, ny = 0, nz = 0, base = 0, levels = 0, nparam = 0, step = 0, version = 0;
    if (st == RSV_OK) {
        const std::string h(line);
        if (h.find("\"format\":\"rsv_unet\"") == std::string::npos || !read_json_int(h, "version", &version) ||
            version != 1 || !read_json_int(h, "nx", &nx) || !read_json_int(h, "ny", &ny) ||
            !read_json_int(h, "nz", &nz) || !read_json_int(h, "base", &base) || !read_json_int(h, "levels", &levels) ||
            !read_json_int(h, "nparam", &nparam) || !read_json_int(h, "adam_step", &step))
            st = RSV_EINVAL;
        // the network must have the stored architecture (grid, width, depth)
        else if (nx != u->nx || ny != u->ny || nz != u->nz || base != u->base || levels != u->L ||
                 nparam != u->nparam || step < 0 || step > (1ll << 30))
            st = RSV_EINVAL;
    }
    if (st == RSV_OK) {
        try {
            buf.resize(3 * (size_t)u->nparam);
        } catch (...) {
            st = RSV_ENOMEM;
        }
    }
    if (st == RSV_OK && (std::fread(buf.data(), sizeof(float), buf.size(), f) != buf.size() || std::fgetc(f) != EOF))
        st = RSV_EINVAL;
    std::fclose(f);
    if (st != RSV_OK) return st;
    float *dst[3] = {u->p, u->m, u->v};
    for (int q = 0; q < 3; ++q)
        RSV_CUDA_TRY(cudaMemcpyAsync(dst[q], buf.data() + q * (size_t)u->nparam, sizeof(float) * u->nparam,
                                     cudaMemcpyHostToDevice, u->st));
    u->adam_t = (int)step;
    u->acts_valid = false;
    RSV_TRY(refresh_bf16(u));
    RSV_CUDA_TRY(cudaStreamSynchronize(u->st));
    return RSV_OK;
}

extern "C" rsv_status rsv_unet_apply(rsv_unet *u, const double *rp, const double *lnk, double *corr) {
    if (!u || !rp || !lnk || !corr) return RSV_EINVAL;
    RSV_TRY(forward(u, rp, lnk, corr));
    return check_err(u);
}

extern "C" rsv_status rsv_unet_train_step(rsv_unet *u, const double *rp, const double *lnk, const double *target,
                                          float lr, double *loss) {
    if (!u || !rp || !lnk || !target) return RSV_EINVAL;
    RSV_TRY(forward(u, rp, lnk, nullptr));
    RSV_TRY(backward(u, target));
    if (lr > 0.0f) {
        u->adam_t += 1;
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 / (1.0 - std::pow(b1, u->adam_t)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(b2, u->adam_t)));
        adam_kernel<<<blocks_for(u->nparam, 256, 2048), 256, 0, u->st>>>(u->p, u->g, u->m, u->v, u->nparam, lr,
                                                                         (float)b1, (float)b2, 1e-8f, c1, c2, u->pw);
        pack_first<<<(u->ch[0] * 64 + 255) / 256, 256, 0, u->st>>>(u->p + u->layers[0].woff, u->ch[0], u->w1c);
        RSV_CUDA_TRY(cudaGetLastError());
        count_launches(2);
    }
    if (loss) RSV_CUDA_TRY(cudaMemcpyAsync(loss, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->st));
    return check_err(u);
}

extern "C" rsv_status rsv_unet_train_batch(rsv_unet *u, int n, const double *const *rp, const double *const *lnk,
                                           const double *const *target, float lr, double *losses) {
    if (!u || n < 0 || (n > 0 && (!rp || !lnk || !target)) || !(lr > 0.0f)) return RSV_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!rp[i] || !lnk[i] || !target[i]) return RSV_EINVAL;
    double *dloss = nullptr;
    if (losses && n > 0) RSV_CUDA_TRY(cudaMallocAsync((void **)&dloss, sizeof(double) * n, u->st));
    rsv_status st = RSV_OK;
    for (int i = 0; i < n && st == RSV_OK; ++i) {
        st = forward(u, rp[i], lnk[i], nullptr);
        if (st == RSV_OK) st = backward(u, target[i]);
        if (st != RSV_OK) break;
        u->adam_t += 1;
        const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, u->adam_t)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, u->adam_t)));
        adam_kernel<<<blocks_for(u->nparam, 256, 2048), 256, 0, u->st>>>(u->p, u->g, u->m, u->v, u->nparam, lr, 0.9f,
                                                                         0.999f, 1e-8f, c1, c2, u->pw);
        pack_first<<<(u->ch[0] * 64 + 255) / 256, 256, 0, u->st>>>(u->p + u->layers[0].woff, u->ch[0], u->w1c);
        count_launches(2);
        if (dloss && cudaMemcpyAsync(dloss + i, u->loss, sizeof(double), cudaMemcpyDeviceToDevice, u->st) != cudaSuccess)
            st = RSV_ECUDA;
        if (cudaGetLastError() != cudaSuccess) st = RSV_ECUDA;
    }
    if (dloss) {
        if (st == RSV_OK &&
            cudaMemcpyAsync(losses, dloss, sizeof(double) * n, cudaMemcpyDeviceToHost, u->st) != cudaSuccess)
            st = RSV_ECUDA;
        cudaFreeAsync(dloss, u->st);
    }
    const rsv_status e = check_err(u);
    return st != RSV_OK ? st : e;
}
