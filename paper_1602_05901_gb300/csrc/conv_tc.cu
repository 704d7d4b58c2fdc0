// 3x3x3 (and 1x1x1) convolutions of the learned pressure stage as implicit
// GEMMs on the tcgen05 tensor cores: BF16 operands staged by TMA, FP32
// accumulators in TMEM, fused epilogues.
//
// Volumes are channels-last BF16, [nz][ny][nx][ld] with the layer's channels
// at the start of each voxel's row of ld values.  A 3x3x3 weight is
// w[co][t][ci] with tap t = 9(dz+1) + 3(dy+1) + (dx+1); the layer computes
// the cross-correlation y[v, co] = sum_t sum_ci w[co,t,ci] x[v + off_t, ci]
// with zeros outside the grid.
//
// Forward (and the input gradient, which is the same correlation with the
// taps mirrored and the channel roles swapped):
//   M = 128 voxels of one tile (a box of bw x bh x bd voxels), N = output
//   channels, K = taps x input channels.  Each K step is one tap and one
//   block of BK channels: TMA copies the tap-shifted box of the input volume
//   (zero fill outside the grid gives the padding exactly) and the matching
//   weight slice; four (BK = 64) or two (BK = 32) MMAs of K = 16 consume it.
// Weight gradient:
//   gw[co][t][ci] = sum_v gy[v, co] x[v + off_t, ci] reduces over voxels, so
//   K = voxels.  Both operands are first copied voxel-major (one row of
//   voxels per channel) into a flat layout padded by one zero slice in z and
//   one zero row in y on each side, so that the dz and dy shifts of a tap are
//   plain offsets of the flat TMA coordinate (zeros arrive at the borders).
//   The dx shift cannot be such an offset (the innermost TMA coordinate must
//   stay 16-byte aligned), so the input is copied three times, pre-shifted by
//   dx = -1, 0, +1.  M = 128 rows of (tap, ci) pairs, N = output channels, K
//   steps of 64 voxels; CTAs split the voxels and write FP32 partial sums
//   that a second kernel adds in a fixed order.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "conv.cuh"
#include "tc.cuh"

namespace rsv {

using namespace tc;

// ------------------------------------------------------------------ host: tensor maps
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// BF16 tensor map of rank r: dims/box innermost first, strides in bytes for dims 1..r-1.
rsv_status make_map(CUtensorMap *m, const void *base, int rank, const uint64_t *dims, const uint64_t *strides,
                    const uint32_t *box, int swz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return RSV_ENOTSUP;
    if (((uintptr_t)base) & 15) return RSV_EINVAL;
    for (int i = 0; i < rank - 1; ++i)
        if (strides[i] % 16) return RSV_EINVAL;
    cuuint64_t d[5], s[4];
    cuuint32_t b[5], e[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        e[i] = 1;
        if (i < rank - 1) s[i] = strides[i];
    }
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void *>(base), d, s, b, e,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? RSV_OK : RSV_EINVAL;
}

constexpr int kStages = 4;
constexpr int kThreads = 128;

__device__ __forceinline__ void raise(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ------------------------------------------------------------------ forward / input-gradient kernel
struct FwdArgs {
    int nx, ny, nz;
    int bw, bh, bd;       // voxel box of one M tile
    int tx, ty;           // tiles along x and y
    int taps, nkb, ci;    // taps (27 or 1), channel blocks per tap, input channels
    int n_total;          // output channels
    const float *bias;    // [n_total] or null
    int relu;
    const __nv_bfloat16 *mask;  // multiply by (mask > 0): [V][ldm] or null
    int ldm;
    __nv_bfloat16 *y;     // [V][ldy] or null
    int ldy;
    float *y32;           // [V][n_total] or null
    int *err;
    uint64_t timeout_ns;
    const int *gate;      // skip the launch when *gate != 0 (may be null)
};

template <int BK, int BN>
struct FwdSmem {
    static constexpr uint32_t A = 128 * BK * 2, B = BN * BK * 2, STAGE = A + B;
    static constexpr uint32_t BARS = kStages * STAGE;
    static constexpr uint32_t BYTES = BARS + 256 + 1024;  // + barriers/slots + alignment slack
};

template <int BK, int BN>
__global__ void __launch_bounds__(kThreads, 1)
    conv_fwd_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const FwdArgs a) {
    if (a.gate && *a.gate) return;  // uniform across the CTA, before any barrier or allocation
    using L = FwdSmem<BK, BN>;
    constexpr int SWZ = BK * 2;  // 128 or 64
    constexpr uint32_t TCOLS = tmem_cols_for(BN);
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t *full = (uint64_t *)(sm + L::BARS);
    uint64_t *empty = full + kStages;
    uint64_t *done = empty + kStages;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    int *flags = (int *)(tmem_slot + 1);  // [0] failed, [1] loads issued, [2] loads consumed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const int x0 = (tile % a.tx) * a.bw;
    const int y0 = ((tile / a.tx) % a.ty) * a.bh;
    const int z0 = (tile / (a.tx * a.ty)) * a.bd;
    const int n0 = blockIdx.y * BN;
    const int nk = a.taps * a.nkb;
    const uint64_t deadline = now_ns() + a.timeout_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        flags[0] = flags[1] = flags[2] = 0;
        fence_mbar_init();
    }
    if (warp == 2) tmem_alloc(tmem_slot, TCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        prefetch_map(&tmA);
        prefetch_map(&tmB);
        const uint32_t bytes = (uint32_t)(a.bw * a.bh * a.bd) * BK * 2 + (uint32_t)BN * BK * 2;
        int kk = 0;
        for (; kk < nk; ++kk) {
            const int s = kk % kStages;
            if (kk >= kStages && !mbar_wait(&empty[s], ((kk / kStages) + 1) & 1, deadline)) {
                flags[0] = 1;
                break;
            }
            const int tap = kk / a.nkb, cb = kk % a.nkb;
            int dz = 0, dy = 0, dx = 0;
            if (a.taps == 27) {
                dz = tap / 9 - 1;
                dy = (tap / 3) % 3 - 1;
                dx = tap % 3 - 1;
            }
            uint8_t *st = sm + s * L::STAGE;
            mbar_expect_tx(&full[s], bytes);
            tma_load_4d(st, &tmA, cb * BK, x0 + dx, y0 + dy, z0 + dz, &full[s]);
            tma_load_2d(st + L::A, &tmB, tap * a.ci + cb * BK, n0, &full[s]);
        }
        flags[1] = kk;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(128, BN);
        int kk = 0;
        for (; kk < nk; ++kk) {
            const int s = kk % kStages;
            if (!mbar_wait(&full[s], (kk / kStages) & 1, deadline)) {
                flags[0] = 1;
                break;
            }
            fence_after_sync();
            const uint32_t sa = smem_u32(sm + s * L::STAGE), sb = sa + L::A;
#pragma unroll
            for (int j = 0; j < BK / 16; ++j)
                mma_bf16(tmem, kmajor_desc(sa + j * 32, SWZ), kmajor_desc(sb + j * 32, SWZ), idesc,
                         (kk > 0 || j > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        flags[2] = kk;
        mma_commit(done);
    }
    __syncwarp();

    // Epilogue: warp w owns TMEM lanes 32w..32w+31, i.e. tile rows (voxels) 32w + lane.
    const bool ok = mbar_wait(done, 0, deadline + a.timeout_ns);
    fence_after_sync();
    const int row = warp * 32 + lane;
    const int rx = row % a.bw, ry = (row / a.bw) % a.bh, rz = row / (a.bw * a.bh);
    const int x = x0 + rx, y = y0 + ry, z = z0 + rz;
    const bool valid = ok && rz < a.bd && x < a.nx && y < a.ny && z < a.nz && !flags[0];
    const int64_t v = ((int64_t)z * a.ny + y) * a.nx + x;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float acc[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc);
        if (!valid) continue;
        const int n = n0 + c0;
        if (a.bias) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] += a.bias[n + i];
        }
        if (a.relu) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = fmaxf(acc[i], 0.0f);
        }
        if (a.mask) {
            const uint4 *mp = (const uint4 *)(a.mask + v * a.ldm + n);
            uint4 mv[2] = {mp[0], mp[1]};
            const __nv_bfloat16 *mb = (const __nv_bfloat16 *)mv;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (!(__bfloat162float(mb[i]) > 0.0f)) acc[i] = 0.0f;
        }
        if (a.y32) {
            float4 *o = (float4 *)(a.y32 + v * a.n_total + n);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
        }
        if (a.y) {
            uint4 ov[2];
            __nv_bfloat162 *ob = (__nv_bfloat162 *)ov;
#pragma unroll
            for (int i = 0; i < 8; ++i) ob[i] = __floats2bfloat162_rn(acc[2 * i], acc[2 * i + 1]);
            uint4 *o = (uint4 *)(a.y + v * a.ldy + n);
            o[0] = ov[0];
            o[1] = ov[1];
        }
    }

    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0 && (flags[0] || !ok)) {
        raise(a.err, RSV_ETIMEOUT);
        // let copies still in flight land before the shared memory is released
        for (int kk = flags[2]; kk < flags[1]; ++kk)
            mbar_wait(&full[kk % kStages], (kk / kStages) & 1, now_ns() + a.timeout_ns);
    }
    __syncthreads();
    if (warp == 2) tmem_dealloc(tmem, TCOLS);
}

// ------------------------------------------------------------------ weight-gradient kernel
struct WgArgs {
    int nchunks, cps;          // 64-voxel K chunks in the padded volume; chunks per split
    int taps, ci, cblk, tpt, ncb;  // tap-group rows: tpt taps x cblk channels; ncb = ci / cblk
    int plane, row;            // flat shift of dz and dy in the padded layout
    int co;                    // output channels (N total)
    float *partial;            // [splits][taps][ci][co]
    int *err;
    uint64_t timeout_ns;
};

template <int BN>
struct WgSmem {
    static constexpr uint32_t A = 128 * 128, B = BN * 128, STAGE = A + B;
    static constexpr uint32_t BARS = kStages * STAGE;
    static constexpr uint32_t BYTES = BARS + 256 + 1024;
};

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    conv_wgrad_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const WgArgs a) {
    using L = WgSmem<BN>;
    constexpr uint32_t TCOLS = tmem_cols_for(BN);
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t *full = (uint64_t *)(sm + L::BARS);
    uint64_t *empty = full + kStages;
    uint64_t *done = empty + kStages;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    int *flags = (int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tg = blockIdx.x / a.ncb, cb = blockIdx.x % a.ncb;
    const int n0 = blockIdx.y * BN;
    const int q0 = blockIdx.z * a.cps;
    const int q1 = min(a.nchunks, q0 + a.cps);
    const int nk = max(0, q1 - q0);
    const int ntap = min(a.tpt, a.taps - tg * a.tpt);
    const uint64_t deadline = now_ns() + a.timeout_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        flags[0] = flags[1] = flags[2] = 0;
        fence_mbar_init();
    }
    if (warp == 2) tmem_alloc(tmem_slot, TCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        prefetch_map(&tmA);
        prefetch_map(&tmB);
        const uint32_t bytes = (uint32_t)ntap * a.cblk * 128 + (uint32_t)BN * 128;
        int kk = 0;
        for (; kk < nk; ++kk) {
            const int s = kk % kStages;
            if (kk >= kStages && !mbar_wait(&empty[s], ((kk / kStages) + 1) & 1, deadline)) {
                flags[0] = 1;
                break;
            }
            const int f0 = (q0 + kk) * 64;
            uint8_t *st = sm + s * L::STAGE;
            mbar_expect_tx(&full[s], bytes);
            for (int g = 0; g < ntap; ++g) {
                const int tap = tg * a.tpt + g;
                int dz = 0, dy = 0, dxi = 0;
                if (a.taps == 27) {
                    dz = tap / 9 - 1;
                    dy = (tap / 3) % 3 - 1;
                    dxi = tap % 3;
                }
                tma_load_3d(st + g * a.cblk * 128, &tmA, f0 + dz * a.plane + dy * a.row, cb * a.cblk, dxi, &full[s]);
            }
            tma_load_2d(st + L::A, &tmB, f0, n0, &full[s]);
        }
        flags[1] = kk;
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(128, BN);
        int kk = 0;
        for (; kk < nk; ++kk) {
            const int s = kk % kStages;
            if (!mbar_wait(&full[s], (kk / kStages) & 1, deadline)) {
                flags[0] = 1;
                break;
            }
            fence_after_sync();
            const uint32_t sa = smem_u32(sm + s * L::STAGE), sb = sa + L::A;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                mma_bf16(tmem, kmajor_desc(sa + j * 32, 128), kmajor_desc(sb + j * 32, 128), idesc,
                         (kk > 0 || j > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        flags[2] = kk;
        mma_commit(done);
    }
    __syncwarp();

    const bool ok = mbar_wait(done, 0, deadline + a.timeout_ns);
    fence_after_sync();
    const int row = warp * 32 + lane;
    const int g = row / a.cblk, c = row % a.cblk;
    const int tap = tg * a.tpt + g;
    const bool valid = ok && g < ntap && !flags[0];
    float *out = a.partial + (((int64_t)blockIdx.z * a.taps + tap) * a.ci + cb * a.cblk + c) * a.co + n0;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float acc[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc);
        if (!valid) continue;
        if (nk == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.0f;
        }
        float4 *o = (float4 *)(out + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
    }

    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0 && (flags[0] || !ok)) {
        raise(a.err, RSV_ETIMEOUT);
        for (int kk = flags[2]; kk < flags[1]; ++kk)
            mbar_wait(&full[kk % kStages], (kk / kStages) & 1, now_ns() + a.timeout_ns);
    }
    __syncthreads();
    if (warp == 2) tmem_dealloc(tmem, TCOLS);
}

// ------------------------------------------------------------------ weight gradient, MN-major operands
// The same reduction over voxels as conv_wgrad_tc, read straight from the
// channels-last tensors: a TMA box of 64 voxels x (32 or 64) channels lands
// in shared memory as 64 rows (K = voxels) of consecutive channels (M or N),
// i.e. an MN-major operand.  Every tap shift (dz, dy, dx) is a plain TMA
// coordinate offset on the voxel axes, with zero fill outside the grid, so no
// copy of the activations is made.
//   A columns: tpt taps x cblk channels = 128 rows of M, in columns of colA
//   (64 or 32) channels; B columns: BN output channels in columns of colB.
struct WgMnArgs {
    int bw, bh, bd;                  // voxel box of one K chunk (bw * bh * bd = 64)
    int kcx, kcy, nchunks, cps;      // chunk grid (x, y; z implied), chunks per split
    int taps, ci, cblk, tpt, ncb, colA;  // ci: channels of the row (tap-shifted) operand
    int co, colB;                    // co: channels of the column operand
    int sgn;                         // +1: rows read at v + off_t; -1: at v - off_t
    float *partial;                  // [splits][taps][ci][co] in the row / column channel roles
    int *err;
    uint64_t timeout_ns;
};

// Pipeline depth per N tile: the deepest ring that still lets two CTAs share an SM.
template <int BN>
struct WgMnSmem {
    static constexpr uint32_t A = 128 * 64 * 2, B = BN * 64 * 2, STAGE = A + B;
    static constexpr int S = STAGE * 4 <= 100 * 1024 ? 4 : STAGE * 3 <= 100 * 1024 ? 3 : 2;
    static constexpr uint32_t BARS = S * STAGE;
    static constexpr uint32_t BYTES = BARS + 256 + 1024;
};

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    conv_wgrad_mn(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmG, const WgMnArgs a) {
    using L = WgMnSmem<BN>;
    constexpr uint32_t TCOLS = tmem_cols_for(BN);
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t *full = (uint64_t *)(sm + L::BARS);
    uint64_t *empty = full + L::S;
    uint64_t *done = empty + L::S;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    int *flags = (int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tg = blockIdx.x / a.ncb, cb = blockIdx.x % a.ncb;
    const int n0 = blockIdx.y * BN;
    const int q0 = blockIdx.z * a.cps;
    const int q1 = min(a.nchunks, q0 + a.cps);
    const int nk = max(0, q1 - q0);
    const int ntap = min(a.tpt, a.taps - tg * a.tpt);
    const int colsA = 128 / a.colA, colsB = BN / a.colB;  // columns per operand
    const int colsPerTap = a.cblk / a.colA;
    const uint32_t rowA = a.colA * 2, rowB = a.colB * 2;  // bytes per K row of a column
    const uint64_t deadline = now_ns() + a.timeout_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < L::S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        flags[0] = flags[1] = flags[2] = 0;
        fence_mbar_init();
    }
    if (warp == 2) tmem_alloc(tmem_slot, TCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        prefetch_map(&tmX);
        prefetch_map(&tmG);
        const uint32_t bytes = (uint32_t)(ntap * colsPerTap) * 64 * rowA + (uint32_t)colsB * 64 * rowB;
        int kk = 0;
        for (; kk < nk; ++kk) {
            const int s = kk % L::S;
            if (kk >= L::S && !mbar_wait(&empty[s], ((kk / L::S) + 1) & 1, deadline)) {
                flags[0] = 1;
                break;
            }
            const int q = q0 + kk;
            const int x0 = (q % a.kcx) * a.bw, y0 = ((q / a.kcx) % a.kcy) * a.bh, z0 = (q / (a.kcx * a.kcy)) * a.bd;
            uint8_t *st = sm + s * L::STAGE;
            mbar_expect_tx(&full[s], bytes);
            for (int g = 0; g < ntap; ++g) {
                const int tap = tg * a.tpt + g;
                int dz = 0, dy = 0, dx = 0;
                if (a.taps == 27) {
                    dz = tap / 9 - 1;
                    dy = (tap / 3) % 3 - 1;
                    dx = tap % 3 - 1;
                }
                for (int j = 0; j < colsPerTap; ++j)
                    tma_load_4d(st + (g * colsPerTap + j) * 64 * rowA, &tmX, cb * a.cblk + j * a.colA,
                                x0 + a.sgn * dx, y0 + a.sgn * dy, z0 + a.sgn * dz, &full[s]);
            }
            for (int j = 0; j < colsB; ++j)
                tma_load_4d(st + L::A + j * 64 * rowB, &tmG, n0 + j * a.colB, x0, y0, z0, &full[s]);
        }
        flags[1] = kk;
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(128, BN, true, true);
        const int swzA = a.colA == 64 ? 128 : 64, swzB = a.colB == 64 ? 128 : 64;
        const uint32_t colbA = 64 * rowA, colbB = 64 * rowB, grpA = 8 * rowA, grpB = 8 * rowB;
        (void)colsA;
        int kk = 0;
        for (; kk < nk; ++kk) {
            const int s = kk % L::S;
            if (!mbar_wait(&full[s], (kk / L::S) & 1, deadline)) {
                flags[0] = 1;
                break;
            }
            fence_after_sync();
            const uint32_t sa = smem_u32(sm + s * L::STAGE), sb = sa + L::A;
#pragma unroll
            for (int j = 0; j < 4; ++j)  // 4 x K = 16 rows = the 64 voxels of the chunk
                mma_bf16(tmem, mnmajor_desc(sa + j * 2 * grpA, swzA, colbA, grpA),
                         mnmajor_desc(sb + j * 2 * grpB, swzB, colbB, grpB), idesc, (kk > 0 || j > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        flags[2] = kk;
        mma_commit(done);
    }
    __syncwarp();

    const bool ok = mbar_wait(done, 0, deadline + a.timeout_ns);
    fence_after_sync();
    const int row = warp * 32 + lane;
    const int g = row / a.cblk, c = row % a.cblk;
    const int tap = tg * a.tpt + g;
    const bool valid = ok && g < ntap && !flags[0];
    float *out = a.partial + (((int64_t)blockIdx.z * a.taps + tap) * a.ci + cb * a.cblk + c) * a.co + n0;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float acc[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc);
        if (!valid) continue;
        if (nk == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.0f;
        }
        float4 *o = (float4 *)(out + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
    }

    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0 && (flags[0] || !ok)) {
        raise(a.err, RSV_ETIMEOUT);
        for (int kk = flags[2]; kk < flags[1]; ++kk)
            mbar_wait(&full[kk % L::S], (kk / L::S) & 1, now_ns() + a.timeout_ns);
    }
    __syncthreads();
    if (warp == 2) tmem_dealloc(tmem, TCOLS);
}

// gb[c] partial sums from the channels-last gradient: CTA b sums its chunk of
// voxels for every channel (lane l owns channels l, l + 32, ...; warps stride
// the voxels), warps added in order.  part[b][co].
__global__ void __launch_bounds__(256) bias_grad_cl(const __nv_bfloat16 *__restrict__ gy, int ld, int co, int64_t V,
                                                    float *__restrict__ part) {
    __shared__ float red[8][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t len = (V + gridDim.x - 1) / gridDim.x;
    const int64_t v0 = blockIdx.x * len, v1 = min(V, v0 + len);
    const int nq = (co + 31) / 32;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t v = v0 + warp;
    for (; v + 24 < v1; v += 32)  // four voxels in flight per warp
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nq && lane + 32 * q < co) {
                const int c = lane + 32 * q;
                const float a0 = __bfloat162float(gy[v * ld + c]), a1 = __bfloat162float(gy[(v + 8) * ld + c]);
                const float a2 = __bfloat162float(gy[(v + 16) * ld + c]), a3 = __bfloat162float(gy[(v + 24) * ld + c]);
                acc[q] += (a0 + a1) + (a2 + a3);
            }
    for (; v < v1; v += 8)
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nq && lane + 32 * q < co) acc[q] += __bfloat162float(gy[v * ld + lane + 32 * q]);
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (lane + 32 * q < co) red[warp][lane + 32 * q] = acc[q];
    __syncthreads();
    for (int c = threadIdx.x; c < co; c += 256) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += red[w][c];
        part[(int64_t)blockIdx.x * co + c] = t;
    }
}
// One warp per channel: lane l adds the blocks l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void bias_grad_cl_final(const float *__restrict__ part, int nblk, int co, float *__restrict__ gb) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= co) return;
    float t = 0.0f;
    for (int b = lane; b < nblk; b += 32) t += part[(int64_t)b * co + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) gb[c] = t;
}

// ------------------------------------------------------------------ helper kernels
// Voxel-major copy of a channels-last volume into the zero-padded flat layout
// of the weight gradient: out[d][c][f], f = ((z+1)(ny+2) + (y+1)) nx + x over
// z in [-1, nz], y in [-1, ny]; out[d][c][f] = x[z, y, x + d - 1, c] when
// nshift = 3 (d = 0, 1, 2), x[z, y, x, c] when nshift = 1; zero outside the grid.
// One CTA per (padded row, 32 channels, 128-voxel chunk of the row): the chunk
// and a one-voxel halo are read once, coalesced along the channels, and
// written nshift times, coalesced along x.
constexpr int kVmChunk = 128;
__global__ void __launch_bounds__(256)
    to_voxel_major(const __nv_bfloat16 *__restrict__ src, int ld, int nch, int nx, int ny, int nz, int nshift,
                   int64_t vpad, __nv_bfloat16 *__restrict__ dst) {
    __shared__ __nv_bfloat16 tile[kVmChunk + 2][33];
    const int row = blockIdx.x;  // padded row index (zp * (ny + 2) + yp)
    const int c0 = blockIdx.y * 32;
    const int x0 = blockIdx.z * kVmChunk;
    const int zp = row / (ny + 2), yp = row - zp * (ny + 2);
    const int z = zp - 1, y = yp - 1;
    const int w = min(kVmChunk, nx - x0);
    const bool real = z >= 0 && z < nz && y >= 0 && y < ny;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    if (real) {
        const int64_t base = ((int64_t)z * ny + y) * nx;
        for (int i = threadIdx.x; i < (w + 2) * 32; i += 256) {
            const int xl = i >> 5, c = i & 31;
            const int x = x0 + xl - 1;
            __nv_bfloat16 v = zero;
            if (x >= 0 && x < nx && c0 + c < nch) v = src[(base + x) * ld + c0 + c];
            tile[xl][c] = v;
        }
    }
    __syncthreads();
    const int64_t f0 = (int64_t)row * nx + x0;
    for (int d = 0; d < nshift; ++d) {
        const int sh = nshift == 3 ? d - 1 : 0;
        for (int i = threadIdx.x; i < 32 * w; i += 256) {
            const int c = i / w, xl = i - c * w;
            if (c0 + c >= nch) continue;
            const __nv_bfloat16 v = real ? tile[xl + 1 + sh][c] : zero;
            dst[((int64_t)d * nch + c0 + c) * vpad + f0 + xl] = v;
        }
    }
}

// gw[co][t][ci] = sum over splits of the partials, in split order.  The partials are
// [s][t][ci][co] (swap = 0), or [s][t][co][ci] (swap = 1: rows were output channels).
__global__ void wgrad_reduce(const float *__restrict__ partial, int splits, int taps, int ci, int co,
                             float *__restrict__ gw, int swap) {
    const int64_t total = (int64_t)taps * ci * co;
    const int ra = swap ? co : ci, rb = swap ? ci : co;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i / ((int64_t)taps * ci));
        const int t = (int)((i / ci) % taps);
        const int c = (int)(i % ci);
        const int row = swap ? o : c, col = swap ? c : o;
        float s = 0.0f;
        for (int q = 0; q < splits; ++q) s += partial[(((int64_t)q * taps + t) * ra + row) * rb + col];
        gw[i] = s;
    }
}

// gb[c] = sum over the padded voxel-major row c (pads are zero): each CTA sums one
// of kBgChunks chunks of a row (fixed tree order), then bias_grad_final adds
// the chunks in order.
constexpr int kBgChunks = 32;
__global__ void __launch_bounds__(256) bias_grad(const __nv_bfloat16 *__restrict__ gyt, int64_t vpad,
                                                 float *__restrict__ part) {
    __shared__ float red[256];
    const __nv_bfloat16 *r = gyt + (int64_t)blockIdx.x * vpad;
    const int64_t len = (vpad + kBgChunks - 1) / kBgChunks;
    const int64_t a = blockIdx.y * len, b = min(vpad, a + len);
    float s = 0.0f;
    for (int64_t f = a + threadIdx.x; f < b; f += 256) s += __bfloat162float(r[f]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * kBgChunks + blockIdx.y] = red[0];
}
__global__ void bias_grad_final(const float *__restrict__ part, int co, float *__restrict__ gb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= co) return;
    float s = 0.0f;
    for (int k = 0; k < kBgChunks; ++k) s += part[c * kBgChunks + k];
    gb[c] = s;
}

// Weights of the input gradient: wt[ci][t][co] = w[co][26 - t][ci].
__global__ void flip_weights(const __nv_bfloat16 *__restrict__ w, int ci, int co, __nv_bfloat16 *__restrict__ wt) {
    const int64_t total = (int64_t)ci * 27 * co;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / (27 * co));
        const int t = (int)((i / co) % 27);
        const int o = (int)(i % co);
        wt[i] = w[((int64_t)o * 27 + (26 - t)) * ci + c];
    }
}

}  // namespace

// ------------------------------------------------------------------ host launchers
namespace {

int pick_bn(int n) {
    for (int b : {256, 192, 128, 96, 64, 32})
        if (n % b == 0) return b;
    return 0;
}

template <typename K>
cudaError_t set_smem(K kernel, uint32_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int BK, int BN>
cudaError_t launch_fwd_t(cudaStream_t st, dim3 grid, const CUtensorMap &ma, const CUtensorMap &mb, const FwdArgs &a) {
    using L = FwdSmem<BK, BN>;
    static cudaError_t attr = set_smem(conv_fwd_tc<BK, BN>, L::BYTES);
    if (attr != cudaSuccess) return attr;
    conv_fwd_tc<BK, BN><<<grid, kThreads, L::BYTES, st>>>(ma, mb, a);
    return cudaGetLastError();
}

template <int BK>
cudaError_t launch_fwd_bk(int bn, cudaStream_t st, dim3 grid, const CUtensorMap &ma, const CUtensorMap &mb,
                          const FwdArgs &a) {
    switch (bn) {
        case 32: return launch_fwd_t<BK, 32>(st, grid, ma, mb, a);
        case 64: return launch_fwd_t<BK, 64>(st, grid, ma, mb, a);
        case 96: return launch_fwd_t<BK, 96>(st, grid, ma, mb, a);
        case 128: return launch_fwd_t<BK, 128>(st, grid, ma, mb, a);
        case 192: return launch_fwd_t<BK, 192>(st, grid, ma, mb, a);
        default: return launch_fwd_t<BK, 256>(st, grid, ma, mb, a);
    }
}

template <int BN>
cudaError_t launch_wg_t(cudaStream_t st, dim3 grid, const CUtensorMap &ma, const CUtensorMap &mb, const WgArgs &a) {
    using L = WgSmem<BN>;
    static cudaError_t attr = set_smem(conv_wgrad_tc<BN>, L::BYTES);
    if (attr != cudaSuccess) return attr;
    conv_wgrad_tc<BN><<<grid, kThreads, L::BYTES, st>>>(ma, mb, a);
    return cudaGetLastError();
}

cudaError_t launch_wg(int bn, cudaStream_t st, dim3 grid, const CUtensorMap &ma, const CUtensorMap &mb,
                      const WgArgs &a) {
    switch (bn) {
        case 32: return launch_wg_t<32>(st, grid, ma, mb, a);
        case 64: return launch_wg_t<64>(st, grid, ma, mb, a);
        case 96: return launch_wg_t<96>(st, grid, ma, mb, a);
        case 128: return launch_wg_t<128>(st, grid, ma, mb, a);
        case 192: return launch_wg_t<192>(st, grid, ma, mb, a);
        default: return launch_wg_t<256>(st, grid, ma, mb, a);
    }
}

template <int BN>
cudaError_t launch_wgmn_t(cudaStream_t st, dim3 grid, const CUtensorMap &ma, const CUtensorMap &mb,
                          const WgMnArgs &a) {
    using L = WgMnSmem<BN>;
    static cudaError_t attr = set_smem(conv_wgrad_mn<BN>, L::BYTES);
    if (attr != cudaSuccess) return attr;
    conv_wgrad_mn<BN><<<grid, kThreads, L::BYTES, st>>>(ma, mb, a);
    return cudaGetLastError();
}

cudaError_t launch_wgmn(int bn, cudaStream_t st, dim3 grid, const CUtensorMap &ma, const CUtensorMap &mb,
                        const WgMnArgs &a) {
    switch (bn) {
        case 32: return launch_wgmn_t<32>(st, grid, ma, mb, a);
        case 64: return launch_wgmn_t<64>(st, grid, ma, mb, a);
        case 96: return launch_wgmn_t<96>(st, grid, ma, mb, a);
        case 128: return launch_wgmn_t<128>(st, grid, ma, mb, a);
        case 192: return launch_wgmn_t<192>(st, grid, ma, mb, a);
        default: return launch_wgmn_t<256>(st, grid, ma, mb, a);
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

struct WgPlan {
    int64_t vpad;
    int nchunks, cblk, tpt, ncb, mtiles, bn, ntiles, splits, cps, nshift;
    size_t xt_bytes, gyt_bytes, part_bytes, bias_bytes;
    bool mn;                 // MN-major path: operands read straight from the channels-last tensors
    bool swap;               // MN path with rows = (tap, output channel): the gradient is the shifted operand
    int bw, bh, bd, kcx, kcy;
};

constexpr int kBiasBlocks = 512;

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

WgPlan wg_plan(ConvVol v, int taps, int ci, int co) {
    WgPlan p{};
    p.bw = std::min(v.nx, 64);
    p.bh = std::min(v.ny, 64 / p.bw);
    p.bd = 64 / (p.bw * p.bh);
    p.mn = p.bw * p.bh * p.bd == 64 && p.bd <= v.nz;
    p.vpad = (int64_t)(v.nz + 2) * (v.ny + 2) * v.nx;
    if (p.mn) {
        p.kcx = (v.nx + p.bw - 1) / p.bw;
        p.kcy = (v.ny + p.bh - 1) / p.bh;
        p.nchunks = p.kcx * p.kcy * ((v.nz + p.bd - 1) / p.bd);
    } else {
        p.nchunks = (int)((p.vpad + 63) / 64);
    }
    // the wider channel count becomes the MMA's N when both operands are read channels-last
    p.swap = p.mn && ci > co;
    const int ra = p.swap ? co : ci, rb = p.swap ? ci : co;
    p.cblk = ra % 128 == 0 ? 128 : ra % 64 == 0 ? 64 : 32;
    p.tpt = 128 / p.cblk;
    p.ncb = ra / p.cblk;
    p.mtiles = ((taps + p.tpt - 1) / p.tpt) * p.ncb;
    p.bn = pick_bn(rb);
    p.ntiles = p.bn ? rb / p.bn : 0;
    const int ctas = std::max(1, p.mtiles * p.ntiles);
    // two resident CTAs per SM: split the voxels so that the grid is at most one wave of 2 x 152
    // (a second, nearly empty wave would double the time)
    int splits = std::max(1, std::min(p.nchunks, (2 * 152) / ctas));
    p.cps = (p.nchunks + splits - 1) / splits;
    p.splits = (p.nchunks + p.cps - 1) / p.cps;
    p.nshift = taps == 27 ? 3 : 1;
    p.xt_bytes = p.mn ? 0 : round256((size_t)p.nshift * ci * p.vpad * 2);
    p.gyt_bytes = p.mn ? 0 : round256((size_t)co * p.vpad * 2);
    p.part_bytes = round256((size_t)p.splits * taps * ci * co * 4);
    p.bias_bytes = round256((size_t)kBiasBlocks * co * 4);
    return p;
}

}  // namespace

rsv_status conv_fwd(cudaStream_t st, ConvVol v, int taps, int ci, int co, const __nv_bfloat16 *x, int ldx,
                    const __nv_bfloat16 *w, const float *bias, int relu, const __nv_bfloat16 *mask, int ldm,
                    __nv_bfloat16 *y, int ldy, float *y32, int *err, uint64_t timeout_ns, const int *gate) {
    if (v.nx <= 0 || v.ny <= 0 || v.nz <= 0 || (taps != 1 && taps != 27) || ci <= 0 || ci % 32 || co <= 0 ||
        co % 32 || !x || !w || (!y && !y32) || ldx < ci || ldx % 8 || (y && (ldy < co || ldy % 8)) ||
        (mask && (ldm < co || ldm % 8)))
        return RSV_EINVAL;
    if (!aligned16(x) || !aligned16(w) || (y && !aligned16(y)) || (y32 && !aligned16(y32)) ||
        (mask && !aligned16(mask)))
        return RSV_EINVAL;
    const int BK = ci % 64 == 0 ? 64 : 32;
    const int BN = pick_bn(co);
    FwdArgs a{};
    a.nx = v.nx;
    a.ny = v.ny;
    a.nz = v.nz;
    a.bw = std::min(v.nx, 128);
    a.bh = std::min(v.ny, 128 / a.bw);
    a.bd = std::min(v.nz, 128 / (a.bw * a.bh));
    a.tx = (v.nx + a.bw - 1) / a.bw;
    a.ty = (v.ny + a.bh - 1) / a.bh;
    const int tz = (v.nz + a.bd - 1) / a.bd;
    a.taps = taps;
    a.nkb = ci / BK;
    a.ci = ci;
    a.n_total = co;
    a.bias = bias;
    a.relu = relu;
    a.mask = mask;
    a.ldm = ldm;
    a.y = y;
    a.ldy = ldy;
    a.y32 = y32;
    a.err = err;
    a.timeout_ns = timeout_ns;
    a.gate = gate;
    CUtensorMap ma, mb;
    {
        const uint64_t dims[4] = {(uint64_t)ci, (uint64_t)v.nx, (uint64_t)v.ny, (uint64_t)v.nz};
        const uint64_t strides[3] = {(uint64_t)ldx * 2, (uint64_t)v.nx * ldx * 2, (uint64_t)v.nx * v.ny * ldx * 2};
        const uint32_t box[4] = {(uint32_t)BK, (uint32_t)a.bw, (uint32_t)a.bh, (uint32_t)a.bd};
        RSV_TRY(make_map(&ma, x, 4, dims, strides, box, BK * 2));
    }
    {
        const uint64_t dims[2] = {(uint64_t)taps * ci, (uint64_t)co};
        const uint64_t strides[1] = {(uint64_t)taps * ci * 2};
        const uint32_t box[2] = {(uint32_t)BK, (uint32_t)BN};
        RSV_TRY(make_map(&mb, w, 2, dims, strides, box, BK * 2));
    }
    const dim3 grid(a.tx * a.ty * tz, co / BN);
    RSV_CUDA_TRY(BK == 64 ? launch_fwd_bk<64>(BN, st, grid, ma, mb, a) : launch_fwd_bk<32>(BN, st, grid, ma, mb, a));
    count_launches(1);
    return RSV_OK;
}

rsv_status conv_flip(cudaStream_t st, int ci, int co, const __nv_bfloat16 *w, __nv_bfloat16 *wt) {
    if (ci <= 0 || co <= 0 || !w || !wt) return RSV_EINVAL;
    const int64_t total = (int64_t)ci * 27 * co;
    flip_weights<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(w, ci, co, wt);
    RSV_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return RSV_OK;
}

size_t conv_wgrad_scratch(ConvVol v, int taps, int ci, int co) {
    const WgPlan p = wg_plan(v, taps, ci, co);
    return p.xt_bytes + p.gyt_bytes + p.part_bytes + p.bias_bytes;
}

rsv_status conv_wgrad(cudaStream_t st, ConvVol v, int taps, int ci, int co, const __nv_bfloat16 *x, int ldx,
                      const __nv_bfloat16 *gy, int ldgy, float *gw, float *gb, void *scratch, int *err,
                      uint64_t timeout_ns) {
    if (v.nx <= 0 || v.ny <= 0 || v.nz <= 0 || v.nx % 8 || (taps != 1 && taps != 27) || ci <= 0 || ci % 32 ||
        co <= 0 || co % 32 || !x || !gy || !gw || !scratch || ldx < ci || ldgy < co)
        return RSV_EINVAL;
    const WgPlan p = wg_plan(v, taps, ci, co);
    if (!aligned16(scratch)) return RSV_EINVAL;
    if (p.mn) {
        if (!aligned16(x) || !aligned16(gy) || ldx % 8 || ldgy % 8) return RSV_EINVAL;
        float *part = (float *)((char *)scratch + p.xt_bytes + p.gyt_bytes);
        float *bpart = (float *)((char *)part + p.part_bytes);
        WgMnArgs a{};
        a.bw = p.bw;
        a.bh = p.bh;
        a.bd = p.bd;
        a.kcx = p.kcx;
        a.kcy = p.kcy;
        a.nchunks = p.nchunks;
        a.cps = p.cps;
        a.taps = taps;
        a.ci = p.swap ? co : ci;
        a.cblk = p.cblk;
        a.tpt = p.tpt;
        a.ncb = p.ncb;
        a.colA = p.cblk >= 64 ? 64 : 32;
        a.co = p.swap ? ci : co;
        a.colB = p.bn % 64 == 0 ? 64 : 32;
        a.sgn = p.swap ? -1 : 1;
        a.partial = part;
        a.err = err;
        a.timeout_ns = timeout_ns;
        // row operand: the tap-shifted one (x, or gy when swapped); column operand: the other
        const __nv_bfloat16 *rowp = p.swap ? gy : x, *colp = p.swap ? x : gy;
        const int rowld = p.swap ? ldgy : ldx, colld = p.swap ? ldx : ldgy;
        CUtensorMap mx, mg;
        {
            const uint64_t dims[4] = {(uint64_t)a.ci, (uint64_t)v.nx, (uint64_t)v.ny, (uint64_t)v.nz};
            const uint64_t strides[3] = {(uint64_t)rowld * 2, (uint64_t)v.nx * rowld * 2,
                                         (uint64_t)v.nx * v.ny * rowld * 2};
            const uint32_t box[4] = {(uint32_t)a.colA, (uint32_t)p.bw, (uint32_t)p.bh, (uint32_t)p.bd};
            RSV_TRY(make_map(&mx, rowp, 4, dims, strides, box, a.colA * 2));
        }
        {
            const uint64_t dims[4] = {(uint64_t)a.co, (uint64_t)v.nx, (uint64_t)v.ny, (uint64_t)v.nz};
            const uint64_t strides[3] = {(uint64_t)colld * 2, (uint64_t)v.nx * colld * 2,
                                         (uint64_t)v.nx * v.ny * colld * 2};
            const uint32_t box[4] = {(uint32_t)a.colB, (uint32_t)p.bw, (uint32_t)p.bh, (uint32_t)p.bd};
            RSV_TRY(make_map(&mg, colp, 4, dims, strides, box, a.colB * 2));
        }
        RSV_CUDA_TRY(launch_wgmn(p.bn, st, dim3(p.mtiles, p.ntiles, p.splits), mx, mg, a));
        const int64_t total = (int64_t)taps * ci * co;
        wgrad_reduce<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(part, p.splits, taps, ci, co,
                                                                                       gw, p.swap ? 1 : 0);
        RSV_CUDA_TRY(cudaGetLastError());
        int n = 2;
        if (gb) {
            const int64_t V = (int64_t)v.nx * v.ny * v.nz;
            bias_grad_cl<<<kBiasBlocks, 256, 0, st>>>(gy, ldgy, co, V, bpart);
            bias_grad_cl_final<<<(co + 7) / 8, 256, 0, st>>>(bpart, kBiasBlocks, co, gb);
            RSV_CUDA_TRY(cudaGetLastError());
            n = 4;
        }
        count_launches(n);
        return RSV_OK;
    }
    __nv_bfloat16 *xt = (__nv_bfloat16 *)scratch;
    __nv_bfloat16 *gyt = (__nv_bfloat16 *)((char *)scratch + p.xt_bytes);
    float *part = (float *)((char *)scratch + p.xt_bytes + p.gyt_bytes);
    const int prow = (v.nz + 2) * (v.ny + 2), xchunks = (v.nx + kVmChunk - 1) / kVmChunk;
    to_voxel_major<<<dim3(prow, ci / 32, xchunks), 256, 0, st>>>(x, ldx, ci, v.nx, v.ny, v.nz, p.nshift, p.vpad, xt);
    RSV_CUDA_TRY(cudaGetLastError());
    to_voxel_major<<<dim3(prow, co / 32, xchunks), 256, 0, st>>>(gy, ldgy, co, v.nx, v.ny, v.nz, 1, p.vpad, gyt);
    RSV_CUDA_TRY(cudaGetLastError());
    CUtensorMap ma, mb;
    {
        const uint64_t dims[3] = {(uint64_t)p.vpad, (uint64_t)ci, (uint64_t)p.nshift};
        const uint64_t strides[2] = {(uint64_t)p.vpad * 2, (uint64_t)ci * p.vpad * 2};
        const uint32_t box[3] = {64u, (uint32_t)p.cblk, 1u};
        RSV_TRY(make_map(&ma, xt, 3, dims, strides, box, 128));
    }
    {
        const uint64_t dims[2] = {(uint64_t)p.vpad, (uint64_t)co};
        const uint64_t strides[1] = {(uint64_t)p.vpad * 2};
        const uint32_t box[2] = {64u, (uint32_t)p.bn};
        RSV_TRY(make_map(&mb, gyt, 2, dims, strides, box, 128));
    }
    WgArgs a{};
    a.nchunks = p.nchunks;
    a.cps = p.cps;
    a.taps = taps;
    a.ci = ci;
    a.cblk = p.cblk;
    a.tpt = p.tpt;
    a.ncb = p.ncb;
    a.plane = (v.ny + 2) * v.nx;
    a.row = v.nx;
    a.co = co;
    a.partial = part;
    a.err = err;
    a.timeout_ns = timeout_ns;
    RSV_CUDA_TRY(launch_wg(p.bn, st, dim3(p.mtiles, p.ntiles, p.splits), ma, mb, a));
    const int64_t total = (int64_t)taps * ci * co;
    wgrad_reduce<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(part, p.splits, taps, ci, co, gw,
                                                                                   0);
    RSV_CUDA_TRY(cudaGetLastError());
    int n = 4;
    if (gb) {
        // the partial sums of the weight gradient are consumed: reuse their buffer
        bias_grad<<<dim3(co, kBgChunks), 256, 0, st>>>(gyt, p.vpad, part);
        bias_grad_final<<<(co + 127) / 128, 128, 0, st>>>(part, co, gb);
        RSV_CUDA_TRY(cudaGetLastError());
        n = 6;
    }
    count_launches(n);
    return RSV_OK;
}

}  // namespace rsv
