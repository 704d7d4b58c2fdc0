// Block ILU(0) triangular sweeps as one persistent launch per sweep.
//
// The forward sweep y_c = D_c^{-1} (r_c - A_{c,-z} y_{-z} - A_{c,-y} y_{-y} -
// A_{c,-x} y_{-x}) has the i+j+k wavefront as its dependency structure
// (Section "Restricted Additive Schwarz Method": L y = b is solved row by
// row).  Instead of one launch per hyperplane, each warp owns a tile of
// 8 (j) x 4 (k) pencils and walks along i.  Lane (a, b) handles cell
// (i = s - a - b, j0 + a, k0 + b) at step s, so the cell's -y and -z
// neighbours inside the tile were computed by lanes (a-1, b) and (a, b-1) one
// step earlier and arrive by warp shuffle; the -x neighbour is the lane's own
// previous result.  Only tile-edge lanes read neighbours owned by other
// warps.  Those values are published by plain stores into an output buffer
// that was pre-filled with a signalling-NaN sentinel: a value is ready when
// it is no longer the sentinel (arithmetic never produces a signalling NaN),
// so no flags or fences are needed.  Edge values are prefetched D steps
// ahead and re-polled (with a time limit) only if still absent.
//
// Each warp's factor data (the three lower or upper blocks and D^{-1} of
// every cell it visits) is packed at setup in exactly the order the warp
// reads it: step-major chunks of 36 x 32 doubles (9216 B).  A TMA bulk copy
// (cp.async.bulk + mbarrier) streams chunk s + NS - 1 into a shared-memory
// ring while step s computes.
//
// The backward sweep z_c = y_c - D_c^{-1} (A_{c,+x} z_{+x} + A_{c,+y} z_{+y} +
// A_{c,+z} z_{+z}) is the mirror image (lane (a, b) visits
// i = nx-1 - (s - (7-a) - (3-b))).  The forward sweep writes the sentinel
// into the output z as it goes and the backward sweep writes it back into
// the scratch y, so both buffers are ready for the next application without
// a separate fill.  Tiles are processed in order of J+K; all warps are
// co-resident (cooperative launch), and a warp only ever waits for tiles
// earlier in that order, so the waits cannot form a cycle.
#include <algorithm>

#include "common.cuh"

namespace rsv {
namespace {

constexpr int TJ = 8, TK = 4;
constexpr int NQ = 36;               // 27 off-diagonal block entries + 9 of D^{-1}
constexpr int NS = 4;                // shared-memory ring stages = prefetch distance
constexpr int CHUNK = NQ * 32;       // values per warp step

// Signalling NaNs: no arithmetic result has these bit patterns.
template <typename T> struct Bits;
template <> struct Bits<double> {
    using U = unsigned long long;
    static constexpr U SENT = 0xFFF4C0DE5A17E7A1ull;
};
template <> struct Bits<float> {
    using U = unsigned int;
    static constexpr U SENT = 0x7FA5C0DEu;
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const double *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const float *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_bits(double *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_bits(float *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long to_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned to_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ double from_bits(unsigned long long v) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ float from_bits(unsigned v) { return __uint_as_float(v); }

template <typename T>
struct SweepArgs {
    int nx, ny, nz, nT, S;
    const int2 *order;         // tile (J, K) per position
    const T *F;                // packed factor chunks [nT][S][36][32]
    const T *in;               // forward: r; backward: y
    T *out;                    // forward: y; backward: z
    T *reset;                  // forward: z (gets the sentinel); backward: y (gets the sentinel)
    const int *done;
    int *status;
    unsigned long long timeout_ns;
};

// Wait until the three components at p are published (not the sentinel).
template <typename T>
__device__ __forceinline__ bool poll3(const T *p, typename Bits<T>::U v[3], uint64_t deadline) {
    for (int e = 0; e < 3; ++e) {
        unsigned spins = 0;
        while (v[e] == Bits<T>::SENT) {
            v[e] = ld_relaxed(p + e);
            if ((++spins & 255u) == 0 && global_timer() > deadline) return false;
        }
    }
    return true;
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(32) ilu_sweep_tiles(SweepArgs<T> P) {
    using U = typename Bits<T>::U;
    constexpr unsigned CHUNK_BYTES = CHUNK * sizeof(T);
    if (P.done && *(volatile const int *)P.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    T *ring = reinterpret_cast<T *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * CHUNK_BYTES);
    const int lane = threadIdx.x;
    const int a = lane & 7, b = lane >> 3;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int64_t sj = nx, sk = (int64_t)nx * ny;
    if (lane == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(&bars[q], 1);
        fence_barrier_init();
    }
    __syncwarp();
    unsigned phase = 0;  // parity bit per ring stage
    const uint64_t deadline = global_timer() + P.timeout_ns;
    bool failed = false;

    unsigned pending = 0;  // ring stages with a bulk copy in flight (tracked by lane 0)
    for (int t = blockIdx.x; t < P.nT && !failed; t += gridDim.x) {
        // forward: tiles in increasing J+K; backward: decreasing (a tile only waits for earlier ones)
        const int tt = FWD ? t : (P.nT - 1 - t);
        const int2 JK = P.order[tt];
        const int j = JK.x * TJ + a, k = JK.y * TK + b;
        const bool jk_ok = (j < ny) && (k < nz);
        const T *Ft = P.F + (size_t)tt * P.S * CHUNK;
        const int S = P.S;
        // direction-dependent geometry
        const int aoff = FWD ? a : (TJ - 1 - a);
        const int boff = FWD ? b : (TK - 1 - b);
        // in-tile neighbour lanes and whether this lane's neighbour lies in another tile
        const int lane_j = FWD ? lane - 1 : lane + 1;      // j -/+ 1
        const int lane_k = FWD ? lane - 8 : lane + 8;      // k -/+ 1
        const bool edge_j = FWD ? (a == 0) : (a == TJ - 1);
        const bool edge_k = FWD ? (b == 0) : (b == TK - 1);
        const bool has_j = FWD ? (j > 0) : (j + 1 < ny);
        const bool has_k = FWD ? (k > 0) : (k + 1 < nz);
        const int64_t dj = FWD ? -sj : sj, dk = FWD ? -sk : sk;

        auto cell_i = [&](int s) { return FWD ? (s - aoff - boff) : (nx - 1 - (s - aoff - boff)); };
        auto cell_valid = [&](int s) {
            const int i = cell_i(s);
            return jk_ok && i >= 0 && i < nx;
        };
        auto cell_of = [&](int s) { return (int64_t)k * sk + (int64_t)j * sj + cell_i(s); };

        // prologue: factor chunks 0..NS-2, vector prefetch for steps 0..NS-1
        if (lane == 0) {
            fence_proxy_async();
            for (int q = 0; q < NS - 1 && q < S; ++q) {
                tma_load_1d(ring + q * CHUNK, Ft + (size_t)q * CHUNK, CHUNK_BYTES, &bars[q]);
                pending |= 1u << q;
            }
        }
        T vin[NS][3];
        U rj[NS][3], rk[NS][3];
#pragma unroll
        for (int u = 0; u < NS; ++u) {
            const bool v = u < S && cell_valid(u);
            const int64_t c = v ? cell_of(u) : 0;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                vin[u][e] = v ? P.in[3 * c + e] : T(0);
                rj[u][e] = (v && edge_j && has_j) ? ld_relaxed(P.out + 3 * (c + dj) + e) : U(0);
                rk[u][e] = (v && edge_k && has_k) ? ld_relaxed(P.out + 3 * (c + dk) + e) : U(0);
            }
        }
        T prev[3] = {T(0), T(0), T(0)};

        for (int s0 = 0; s0 < S; s0 += NS) {
#pragma unroll
            for (int u = 0; u < NS; ++u) {
                const int s = s0 + u;
                if (s >= S) break;
                // refill the stage freed by step s-1
                if (lane == 0 && s + NS - 1 < S) {
                    const int st = (u + NS - 1) % NS;
                    fence_proxy_async();
                    tma_load_1d(ring + st * CHUNK, Ft + (size_t)(s + NS - 1) * CHUNK, CHUNK_BYTES, &bars[st]);
                    pending |= 1u << st;
                }
                const bool valid = cell_valid(s);
                const int64_t c = valid ? cell_of(s) : 0;
                // neighbours: shuffles of the previous step's results
                T nj[3], nk[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const T sjv = __shfl_sync(0xffffffffu, prev[e], lane_j & 31);
                    const T skv = __shfl_sync(0xffffffffu, prev[e], lane_k & 31);
                    nj[e] = has_j ? sjv : T(0);
                    nk[e] = has_k ? skv : T(0);
                }
                if (valid && edge_j && has_j) {
                    if (!poll3(P.out + 3 * (c + dj), rj[u], deadline)) failed = true;
#pragma unroll
                    for (int e = 0; e < 3; ++e) nj[e] = from_bits(rj[u][e]);
                }
                if (valid && edge_k && has_k) {
                    if (!poll3(P.out + 3 * (c + dk), rk[u], deadline)) failed = true;
#pragma unroll
                    for (int e = 0; e < 3; ++e) nk[e] = from_bits(rk[u][e]);
                }
                // factor chunk of this step
                {
                    unsigned spins = 0;
                    bool landed = true;
                    while (!mbar_try_wait(&bars[u], (phase >> u) & 1u)) {
                        if ((++spins & 1023u) == 0 && global_timer() > deadline) {
                            failed = true;
                            landed = false;
                            break;
                        }
                    }
                    if (landed) {
                        phase ^= 1u << u;
                        pending &= ~(1u << u);
                    }
                }
                const T *Fs = ring + u * CHUNK + lane;
                const bool has_i = FWD ? (cell_i(s) > 0) : (cell_i(s) < nx - 1);
                T own[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) own[e] = has_i ? prev[e] : T(0);
                // slots: FWD  [0] -z  [1] -y  [2] -x ;  BWD  [0] +x  [1] +y  [2] +z
                const T *xs0 = FWD ? nk : own;
                const T *xs2 = FWD ? own : nk;
                T acc[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    T sum = T(0);
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        sum = fma(Fs[(0 * 9 + 3 * e + f) * 32], xs0[f], sum);
                        sum = fma(Fs[(1 * 9 + 3 * e + f) * 32], nj[f], sum);
                        sum = fma(Fs[(2 * 9 + 3 * e + f) * 32], xs2[f], sum);
                    }
                    acc[e] = FWD ? (vin[u][e] - sum) : sum;
                }
                T res[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const T d = Fs[(27 + 3 * e) * 32] * acc[0] + Fs[(28 + 3 * e) * 32] * acc[1] +
                                Fs[(29 + 3 * e) * 32] * acc[2];
                    res[e] = FWD ? d : (vin[u][e] - d);
                }
                if (valid) {
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        st_relaxed_bits(P.out + 3 * c + e, to_bits(res[e]));
                        st_relaxed_bits(P.reset + 3 * c + e, Bits<T>::SENT);
                    }
                }
#pragma unroll
                for (int e = 0; e < 3; ++e) prev[e] = valid ? res[e] : T(0);
                // prefetch the vectors of step s + NS into this slot
                {
                    const int sn = s + NS;
                    const bool vn = sn < S && cell_valid(sn);
                    const int64_t cn = vn ? cell_of(sn) : 0;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        vin[u][e] = vn ? P.in[3 * cn + e] : T(0);
                        rj[u][e] = (vn && edge_j && has_j) ? ld_relaxed(P.out + 3 * (cn + dj) + e) : U(0);
                        rk[u][e] = (vn && edge_k && has_k) ? ld_relaxed(P.out + 3 * (cn + dk) + e) : U(0);
                    }
                }
                __syncwarp();
            }
            if (__any_sync(0xffffffffu, failed)) {
                failed = true;
                break;
            }
        }
    }
    if (failed) {
        if (lane == 0) atomicCAS(P.status, 0, (int)RSV_ETIMEOUT);
        // let copies still in flight land before the CTA exits (bounded)
        if (lane == 0) {
            const uint64_t limit = global_timer() + 1000000000ull;
            for (int q = 0; q < NS; ++q)
                if (pending & (1u << q))
                    while (!mbar_try_wait(&bars[q], (phase >> q) & 1u) && global_timer() < limit) {
                    }
        }
        __syncwarp();
    }
}

// Pack the factor into warp-step chunks.  One thread per (tile, step, lane).
// Block values come from `v` (FP64, or the FP32 copy for mixed precision);
// D^{-1} from the FP64 factor; both are stored as T.
template <typename T, typename Tv>
__global__ void pack_tiles(int nx, int ny, int nz, int nT, int S, const int2 *__restrict__ order,
                           const int32_t *__restrict__ rp, const Tv *__restrict__ v,
                           const double *__restrict__ dinv, T *__restrict__ Ff, T *__restrict__ Fb) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nT * S * 32;
    if (gid >= total) return;
    const int lane = (int)(gid & 31);
    const int s = (int)((gid >> 5) % S);
    const int t = (int)((gid >> 5) / S);
    const int a = lane & 7, b = lane >> 3;
    const int2 JK = order[t];
    const int j = JK.x * TJ + a, k = JK.y * TK + b;
    for (int dir = 0; dir < 2; ++dir) {
        const bool fwd = dir == 0;
        const int i = fwd ? (s - a - b) : (nx - 1 - (s - (TJ - 1 - a) - (TK - 1 - b)));
        T *out = (fwd ? Ff : Fb) + ((size_t)t * S + s) * CHUNK + lane;
        const bool valid = j < ny && k < nz && i >= 0 && i < nx;
        if (!valid) {
            for (int q = 0; q < NQ; ++q) out[q * 32] = T(0);
            continue;
        }
        const int64_t c = (int64_t)k * nx * ny + (int64_t)j * nx + i;
        // slots of the row: -z, -y, -x, self, +x, +y, +z (absent faces skipped)
        int q = 0, mz = -1, my = -1, mx = -1, px = -1, py = -1, pz = -1;
        if (k > 0) mz = q++;
        if (j > 0) my = q++;
        if (i > 0) mx = q++;
        q++;
        if (i < nx - 1) px = q++;
        if (j < ny - 1) py = q++;
        if (k < nz - 1) pz = q++;
        const int sl[3] = {fwd ? mz : px, fwd ? my : py, fwd ? mx : pz};
        for (int blk = 0; blk < 3; ++blk)
            for (int e = 0; e < 9; ++e)
                out[(blk * 9 + e) * 32] = sl[blk] >= 0 ? (T)v[9 * ((int64_t)rp[c] + sl[blk]) + e] : T(0);
        for (int e = 0; e < 9; ++e) out[(27 + e) * 32] = (T)dinv[9 * c + e];
    }
}

template <typename T>
__global__ void fill_sentinel(int64_t n, T *p) {
    using U = typename Bits<T>::U;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<U *>(p)[i] = Bits<T>::SENT;
}

}  // namespace

template <typename T>
cudaError_t tiles_setup(const rsv_mat *A, const double *dinv, IluTiles *T_) {
    IluTiles *Tl = T_;
    const int nx = A->nx, ny = A->ny, nz = A->nz;
    const int nTJ = (ny + TJ - 1) / TJ, nTK = (nz + TK - 1) / TK;
    const int nT = nTJ * nTK;
    const int S = nx + TJ + TK - 2;
    const size_t chunk_bytes = CHUNK * sizeof(T);
    cudaError_t e = cudaSuccess;
    if (!Tl->Ff || Tl->nT != nT || Tl->S != S || Tl->elem != (int)sizeof(T)) {
        free_tiles(Tl);
        std::vector<int2> order;
        order.reserve(nT);
        for (int d = 0; d <= nTJ + nTK - 2; ++d)
            for (int J = 0; J < nTJ; ++J) {
                const int K = d - J;
                if (K >= 0 && K < nTK) order.push_back(make_int2(J, K));
            }
        Tl->nT = nT;
        Tl->S = S;
        Tl->elem = (int)sizeof(T);
        const size_t fbytes = (size_t)nT * S * chunk_bytes;
        if ((e = cudaMalloc(&Tl->Ff, fbytes)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&Tl->Fb, fbytes)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void **)&Tl->order, sizeof(int2) * nT)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&Tl->scratch, sizeof(T) * 3 * std::max<int64_t>(A->nb, 1))) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(Tl->order, order.data(), sizeof(int2) * nT, cudaMemcpyHostToDevice, A->stream)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(A->stream)) != cudaSuccess) return e;
        int dev = 0, sms = 0, per_f = 0, per_b = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t smem = NS * chunk_bytes + NS * sizeof(uint64_t);
        if ((e = cudaFuncSetAttribute((const void *)ilu_sweep_tiles<T, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute((const void *)ilu_sweep_tiles<T, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, ilu_sweep_tiles<T, true>, 32, smem)) !=
                cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_b, ilu_sweep_tiles<T, false>, 32, smem)) !=
                cudaSuccess)
            return e;
        Tl->grid = std::max(1, std::min(nT, sms * std::min(per_f, per_b)));
        Tl->smem = smem;
    }
    const int64_t total = (int64_t)nT * S * 32;
    const unsigned g = (unsigned)((total + 255) / 256);
    rsv::count_launches(1);
    if (sizeof(T) == 8)
        pack_tiles<T, double><<<g, 256, 0, A->stream>>>(nx, ny, nz, nT, S, Tl->order, A->d_rp, A->d_v, dinv,
                                                        (T *)Tl->Ff, (T *)Tl->Fb);
    else
        pack_tiles<T, float><<<g, 256, 0, A->stream>>>(nx, ny, nz, nT, S, Tl->order, A->d_rp, A->d_v32, dinv,
                                                       (T *)Tl->Ff, (T *)Tl->Fb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return reset_tiles_scratch(A, Tl);
}

cudaError_t reset_tiles_scratch(const rsv_mat *A, IluTiles *Tl) {
    const int64_t n = 3 * A->nb;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    rsv::count_launches(1);
    if (Tl->elem == 8)
        fill_sentinel<double><<<g, 256, 0, A->stream>>>(n, (double *)Tl->scratch);
    else
        fill_sentinel<float><<<g, 256, 0, A->stream>>>(n, (float *)Tl->scratch);
    return cudaGetLastError();
}

void free_tiles(IluTiles *Tl) {
    if (Tl->Ff) cudaFree(Tl->Ff);
    if (Tl->Fb) cudaFree(Tl->Fb);
    if (Tl->order) cudaFree(Tl->order);
    if (Tl->scratch) cudaFree(Tl->scratch);
    *Tl = IluTiles();
}

template <typename T>
cudaError_t launch_ilu_apply_tiles(const rsv_mat *A, const IluTiles &Tl, const T *r, T *z, const int *done,
                                   int *status, unsigned long long timeout_ns) {
    SweepArgs<T> f{A->nx, A->ny, A->nz, Tl.nT, Tl.S, Tl.order, (const T *)Tl.Ff, r, (T *)Tl.scratch, z,
                   done, status, timeout_ns};
    SweepArgs<T> bw{A->nx, A->ny, A->nz, Tl.nT, Tl.S, Tl.order, (const T *)Tl.Fb, (const T *)Tl.scratch, z,
                    (T *)Tl.scratch, done, status, timeout_ns};
    void *fa[] = {&f};
    void *ba[] = {&bw};
    rsv::count_launches(2);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)ilu_sweep_tiles<T, true>, dim3(Tl.grid), dim3(32), fa,
                                                Tl.smem, A->stream);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)ilu_sweep_tiles<T, false>, dim3(Tl.grid), dim3(32), ba, Tl.smem,
                                       A->stream);
}

template cudaError_t tiles_setup<double>(const rsv_mat *, const double *, IluTiles *);
template cudaError_t tiles_setup<float>(const rsv_mat *, const double *, IluTiles *);
template cudaError_t launch_ilu_apply_tiles<double>(const rsv_mat *, const IluTiles &, const double *, double *,
                                                    const int *, int *, unsigned long long);
template cudaError_t launch_ilu_apply_tiles<float>(const rsv_mat *, const IluTiles &, const float *, float *,
                                                   const int *, int *, unsigned long long);

}  // namespace rsv
