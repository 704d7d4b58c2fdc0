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
// previous result.
//
// Everything else a step needs arrives through shared-memory rings filled by
// TMA bulk copies (cp.async.bulk + mbarrier): a deep data ring (NSD - 1 steps
// ahead, hiding HBM latency) and a shallow edge ring (NSE - 1 steps ahead):
//   * the factor row of each lane (three off-diagonal blocks and D^{-1}, 36
//     values, packed at setup in exactly the order the warp reads them);
//   * the input vector, gathered into the same tile order before the sweep;
//   * the values of neighbouring tiles' edge cells.  A tile publishes the
//     results of its last j-row and last k-layer into small per-tile edge
//     buffers indexed by the step at which the neighbour will need them.  The
//     buffers hold a signalling-NaN sentinel until written (arithmetic never
//     produces one), so a consumer that finds the sentinel in its staged copy
//     re-reads the value from global memory until it appears (bounded by a
//     time limit that ends the sweep with RSV_ETIMEOUT).
//
// The backward sweep z_c = y_c - D_c^{-1} (A_{c,+x} z_{+x} + A_{c,+y} z_{+y} +
// A_{c,+z} z_{+z}) is the mirror image (lane (a, b) visits
// i = nx-1 - (s - (7-a) - (3-b))).  The forward sweep writes y straight into
// the tile order the backward sweep reads (at forward step s every lane's
// cell is visited at backward step S-1-s), so y never exists in natural
// order; the backward sweep writes z in natural order.
//
// Tiles are processed in order of J+K (backward: reverse order); all warps
// are co-resident (cooperative launch), and a warp only ever waits for tiles
// earlier in its order, so the waits cannot form a cycle.
#include <algorithm>

#include "common.cuh"

namespace rsv {
namespace {

constexpr int TJ = 8, TK = 4;
// Edge ring stages: neighbour values are copied NSE - 1 steps ahead.  Each step of
// look-ahead is a step of lag per tile hand-off on the sweep's critical path, so
// the ring is one step deep (measured on 100x100x50: 546 us per FP32 apply with
// two steps of look-ahead, 480 us with one; plain register loads one step ahead,
// without TMA, were slower still: 577 us).
constexpr int NSE = 2;

template <typename T> struct Bits;
template <> struct Bits<double> {
    using U = unsigned long long;
    static constexpr U SENT = 0xFFF4C0DE5A17E7A1ull;  // signalling NaN
    static constexpr int NQP = 38;                    // padded factor row: conflict-free 16-byte reads
    static constexpr int NSD = 6;                     // data ring stages (copies NSD - 1 steps ahead)
};
template <> struct Bits<float> {
    using U = unsigned int;
    static constexpr U SENT = 0x7FA5C0DEu;
    static constexpr int NQP = 36;
    static constexpr int NSD = 10;
};

// Data ring stage: factor [32][NQP] | vector [32][4].  Edge ring stage: edge j [4][4] | edge k [8][4].
// The data ring runs deep (hides HBM latency); the edge ring runs shallow, so that
// neighbour values are copied as late as possible and are mostly already published.
template <typename T> struct Stage {
    static constexpr int F = 32 * Bits<T>::NQP;
    static constexpr int V = 32 * 4;
    static constexpr int EJ = TK * 4;
    static constexpr int EK = TJ * 4;
    static constexpr int SIZE = F + V;
    static constexpr int ESIZE = EJ + EK;
    static constexpr unsigned FB = F * sizeof(T), VB = V * sizeof(T), EJB = EJ * sizeof(T), EKB = EK * sizeof(T);
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
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
__device__ __forceinline__ void st_relaxed(double *p, double v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(__double_as_longlong(v)) : "memory");
}
__device__ __forceinline__ void st_relaxed(float *p, float v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(__float_as_uint(v)) : "memory");
}
__device__ __forceinline__ unsigned long long bits_of(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned bits_of(float v) { return __float_as_uint(v); }
__device__ __forceinline__ double value_of(unsigned long long v) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ float value_of(unsigned v) { return __uint_as_float(v); }

template <typename T>
struct SweepArgs {
    int nT;                    // tiles of all grids
    const TileSys *tsys;       // per grid
    const int *tile_sys;       // position -> grid
    const int64_t *tile_row0;  // position -> first step row of the tile in the packed arrays
    const int2 *order;         // position -> tile (J, K) inside its grid
    const int *pos_of;         // grid's poff + J * nTK + K -> position
    const T *F;          // factor rows [nT][S][32][NQP]
    const T *V;          // input vector in tile order [nT][S][32][4]
    T *Vnext;            // forward: y in backward tile order [nT][S][32][4]; backward: null
    T *z;                // backward: output in natural order; forward: null
    T *EJ, *EK;          // edge buffers this sweep publishes [nT][S][TK][4], [nT][S][TJ][4]
    T *EJnext, *EKnext;  // forward: the backward sweep's edge buffers (reset to the sentinel)
    const int *done;
    int *status;
    unsigned long long timeout_ns;
};

// Re-read a staged neighbour value that was still the sentinel.
template <typename T>
__device__ __forceinline__ bool poll3(const T *g, T v[3], uint64_t deadline) {
    using U = typename Bits<T>::U;
    unsigned spins = 0;
    for (;;) {
        U b0 = bits_of(v[0]), b1 = bits_of(v[1]), b2 = bits_of(v[2]);
        if (b0 != Bits<T>::SENT && b1 != Bits<T>::SENT && b2 != Bits<T>::SENT) return true;
        b0 = ld_relaxed(g);
        b1 = ld_relaxed(g + 1);
        b2 = ld_relaxed(g + 2);
        v[0] = value_of(b0);
        v[1] = value_of(b1);
        v[2] = value_of(b2);
        if ((++spins & 63u) == 0 && global_timer() > deadline) return false;
    }
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(32) ilu_sweep_tiles(SweepArgs<T> P) {
    using St = Stage<T>;
    constexpr int NQP = Bits<T>::NQP;
    constexpr int NSD = Bits<T>::NSD;
    if (P.done && *(volatile const int *)P.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    T *ring = reinterpret_cast<T *>(smem);                       // NSD data stages
    T *ering = ring + NSD * St::SIZE;                            // NSE edge stages
    uint64_t *bars = reinterpret_cast<uint64_t *>(ering + NSE * St::ESIZE);  // NSD data + NSE edge barriers
    uint64_t *ebars = bars + NSD;
    const int lane = threadIdx.x;
    const int a = lane & 7, b = lane >> 3;
    if (lane == 0) {
        for (int q = 0; q < NSD + NSE; ++q) mbar_init(&bars[q], 1);
        fence_barrier_init();
    }
    __syncwarp();
    unsigned phase = 0, pending = 0;  // bit q: data stage q; bit NSD + q: edge stage q
    const uint64_t deadline = global_timer() + P.timeout_ns;
    bool failed = false;

    for (int t = blockIdx.x; t < P.nT && !failed; t += gridDim.x) {
        const int tt = FWD ? t : (P.nT - 1 - t);
        const TileSys G = P.tsys[P.tile_sys[tt]];
        const int nx = G.nx, ny = G.ny, nz = G.nz, S = G.S, nTJ = G.nTJ, nTK = G.nTK;
        const int2 JK = P.order[tt];
        // producers of this tile's edge inputs (same grid)
        const int pj = FWD ? (JK.x > 0 ? P.pos_of[G.poff + (JK.x - 1) * nTK + JK.y] : -1)
                           : (JK.x + 1 < nTJ ? P.pos_of[G.poff + (JK.x + 1) * nTK + JK.y] : -1);
        const int pk = FWD ? (JK.y > 0 ? P.pos_of[G.poff + JK.x * nTK + JK.y - 1] : -1)
                           : (JK.y + 1 < nTK ? P.pos_of[G.poff + JK.x * nTK + JK.y + 1] : -1);
        const int j = JK.x * TJ + a, k = JK.y * TK + b;
        const bool jk_ok = (j < ny) && (k < nz);
        const bool has_j = FWD ? (j > 0) : (j + 1 < ny);
        const bool has_k = FWD ? (k > 0) : (k + 1 < nz);
        const bool edge_j = FWD ? (a == 0) : (a == TJ - 1);
        const bool edge_k = FWD ? (b == 0) : (b == TK - 1);
        const bool pub_j = FWD ? (a == TJ - 1) : (a == 0);  // this lane's results feed the next tile in j
        const bool pub_k = FWD ? (b == TK - 1) : (b == 0);
        const int lane_j = (FWD ? lane - 1 : lane + 1) & 31;
        const int lane_k = (FWD ? lane - 8 : lane + 8) & 31;
        const int off = FWD ? (a + b) : ((TJ - 1 - a) + (TK - 1 - b));
        const int64_t base = G.cell0 + (int64_t)k * nx * ny + (int64_t)j * nx;
        const size_t tile0 = (size_t)P.tile_row0[tt];
        const size_t rowj = pj >= 0 ? (size_t)P.tile_row0[pj] : 0, rowk = pk >= 0 ? (size_t)P.tile_row0[pk] : 0;
        const T *Ft = P.F + tile0 * St::F;
        const T *Vt = P.V + tile0 * St::V;
        const T *EJsrc = pj >= 0 ? P.EJ + rowj * St::EJ : nullptr;
        const T *EKsrc = pk >= 0 ? P.EK + rowk * St::EK : nullptr;
        if (FWD) {
            // this tile's backward-sweep edge buffers start at the sentinel
            using U = typename Bits<T>::U;
            U *ej = reinterpret_cast<U *>(P.EJnext + tile0 * St::EJ);
            U *ek = reinterpret_cast<U *>(P.EKnext + tile0 * St::EK);
            for (int q = lane; q < S * St::EJ; q += 32) ej[q] = Bits<T>::SENT;
            for (int q = lane; q < S * St::EK; q += 32) ek[q] = Bits<T>::SENT;
        }
        const bool edges = pj >= 0 || pk >= 0;
        const unsigned edge_bytes = (pj >= 0 ? St::EJB : 0u) + (pk >= 0 ? St::EKB : 0u);
        auto issue_at = [&](int s, int st) {  // step s into data stage st (= s % NSD)
            T *dst = ring + st * St::SIZE;
            mbar_expect(&bars[st], St::FB + St::VB);
            tma_load_1d(dst, Ft + (size_t)s * St::F, St::FB, &bars[st]);
            tma_load_1d(dst + St::F, Vt + (size_t)s * St::V, St::VB, &bars[st]);
            pending |= 1u << st;
        };
        auto issue_edges_at = [&](int s, int st) {  // step s into edge stage st (= s % NSE)
            if (!edges) return;
            T *dst = ering + st * St::ESIZE;
            mbar_expect(&ebars[st], edge_bytes);
            if (pj >= 0) tma_load_1d(dst, EJsrc + (size_t)s * St::EJ, St::EJB, &ebars[st]);
            if (pk >= 0) tma_load_1d(dst + St::EJ, EKsrc + (size_t)s * St::EK, St::EKB, &ebars[st]);
            pending |= 1u << (NSD + st);
        };
        auto wait_stage = [&](uint64_t *bar, int bit) {
            unsigned spins = 0;
            while (!mbar_try_wait(bar, (phase >> bit) & 1u)) {
                if ((++spins & 1023u) == 0 && global_timer() > deadline) {
                    failed = true;
                    return;
                }
            }
            phase ^= 1u << bit;
            pending &= ~(1u << bit);
        };
        if (lane == 0) {
            fence_proxy_async();
            for (int q = 0; q < NSD - 1 && q < S; ++q) issue_at(q, q);
            for (int q = 0; q < NSE - 1 && q < S; ++q) issue_edges_at(q, q);
        }
        T prev[3] = {T(0), T(0), T(0)};
        // Per-step state kept incrementally, so that a step holds no division and no 64-bit
        // index product: the ring stages of this step and of the next copies, the cell index
        // along x, and the addresses this lane reads or writes.
        int st = 0, est = 0;
        int ist = (NSD - 1) % NSD, iest = (NSE - 1) % NSE;
        int i = FWD ? -off : (nx - 1 + off);
        T *yout = FWD ? P.Vnext + ((tile0 + (S - 1)) * 32 + lane) * 4 : P.z + 3 * (base + i);
        const ptrdiff_t ystep = FWD ? -(ptrdiff_t)(32 * 4) : -3;
        T *pubj = P.EJ + ((ptrdiff_t)tile0 - (TJ - 1)) * St::EJ + b * 4;  // row of step s - (TJ - 1)
        T *pubk = P.EK + ((ptrdiff_t)tile0 - (TK - 1)) * St::EK + a * 4;
        const T *pollj = P.EJ + rowj * St::EJ + b * 4;  // the j producer's row of step s
        const T *pollk = P.EK + rowk * St::EK + a * 4;

        for (int s0 = 0; s0 < S; s0 += 4) {
#pragma unroll 1
            for (int s = s0; s < s0 + 4 && s < S; ++s) {
                // lane 0 refills the stages the previous step used (every lane finished that
                // step: __syncwarp at its end)
                if (lane == 0) {
                    fence_proxy_async();
                    if (s + NSD - 1 < S) issue_at(s + NSD - 1, ist);
                    if (s + NSE - 1 < S) issue_edges_at(s + NSE - 1, iest);
                }
                ist = ist + 1 == NSD ? 0 : ist + 1;
                iest = iest + 1 == NSE ? 0 : iest + 1;
                const bool valid = jk_ok && i >= 0 && i < nx;
                const bool has_i = FWD ? (i > 0) : (i < nx - 1);
                // in-tile neighbours: previous step's results of the adjacent lanes
                T nj[3], nk[3], own[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const T vj = __shfl_sync(0xffffffffu, prev[e], lane_j);
                    const T vk = __shfl_sync(0xffffffffu, prev[e], lane_k);
                    nj[e] = has_j ? vj : T(0);
                    nk[e] = has_k ? vk : T(0);
                    own[e] = has_i ? prev[e] : T(0);
                }
                // wait for this step's stages
                wait_stage(&bars[st], st);
                if (edges) wait_stage(&ebars[est], NSD + est);
                const T *stg = ring + st * St::SIZE;
                const T *estg = ering + est * St::ESIZE;
                st = st + 1 == NSD ? 0 : st + 1;
                est = est + 1 == NSE ? 0 : est + 1;
                if (valid && edge_j && has_j) {
                    const T *e4 = estg + b * 4;
                    T v3[3] = {e4[0], e4[1], e4[2]};
                    if (!poll3(pollj, v3, deadline)) failed = true;
                    nj[0] = v3[0];
                    nj[1] = v3[1];
                    nj[2] = v3[2];
                }
                if (valid && edge_k && has_k) {
                    const T *e4 = estg + St::EJ + a * 4;
                    T v3[3] = {e4[0], e4[1], e4[2]};
                    if (!poll3(pollk, v3, deadline)) failed = true;
                    nk[0] = v3[0];
                    nk[1] = v3[1];
                    nk[2] = v3[2];
                }
                pollj += St::EJ;
                pollk += St::EK;
                // factor row and input of this lane
                T f[NQP];
                {
                    const T *row = stg + lane * NQP;
                    if (sizeof(T) == 4) {
#pragma unroll
                        for (int q = 0; q < 9; ++q) {
                            const float4 v4 = reinterpret_cast<const float4 *>(row)[q];
                            f[4 * q] = v4.x;
                            f[4 * q + 1] = v4.y;
                            f[4 * q + 2] = v4.z;
                            f[4 * q + 3] = v4.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 18; ++q) {
                            const double2 v2 = reinterpret_cast<const double2 *>(row)[q];
                            f[2 * q] = v2.x;
                            f[2 * q + 1] = v2.y;
                        }
                    }
                }
                T vin[3];
                {
                    const T *v4 = stg + St::F + lane * 4;
                    vin[0] = v4[0];
                    vin[1] = v4[1];
                    vin[2] = v4[2];
                }
                // slots: forward [0] -z [1] -y [2] -x ; backward [0] +x [1] +y [2] +z
                const T *x0 = FWD ? nk : own;
                const T *x2 = FWD ? own : nk;
                T acc[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    T p0 = f[3 * e] * x0[0];
                    T p1 = f[9 + 3 * e] * nj[0];
                    T p2 = f[18 + 3 * e] * x2[0];
                    p0 = fma(f[3 * e + 1], x0[1], p0);
                    p1 = fma(f[9 + 3 * e + 1], nj[1], p1);
                    p2 = fma(f[18 + 3 * e + 1], x2[1], p2);
                    p0 = fma(f[3 * e + 2], x0[2], p0);
                    p1 = fma(f[9 + 3 * e + 2], nj[2], p1);
                    p2 = fma(f[18 + 3 * e + 2], x2[2], p2);
                    const T sum = (p0 + p1) + p2;
                    acc[e] = FWD ? (vin[e] - sum) : sum;
                }
                T res[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const T d = fma(f[27 + 3 * e + 2], acc[2], fma(f[27 + 3 * e + 1], acc[1], f[27 + 3 * e] * acc[0]));
                    res[e] = FWD ? d : (vin[e] - d);
                }
                if (valid) {
                    yout[0] = res[0];
                    yout[1] = res[1];
                    yout[2] = res[2];
                    if (pub_j && s >= TJ - 1) {
                        st_relaxed(pubj, res[0]);
                        st_relaxed(pubj + 1, res[1]);
                        st_relaxed(pubj + 2, res[2]);
                    }
                    if (pub_k && s >= TK - 1) {
                        st_relaxed(pubk, res[0]);
                        st_relaxed(pubk + 1, res[1]);
                        st_relaxed(pubk + 2, res[2]);
                    }
                }
                yout += ystep;
                pubj += St::EJ;
                pubk += St::EK;
                i += FWD ? 1 : -1;
#pragma unroll
                for (int e = 0; e < 3; ++e) prev[e] = valid ? res[e] : T(0);
                __syncwarp();
            }
            if (__any_sync(0xffffffffu, failed)) {
                failed = true;
                break;
            }
        }
    }
    if (failed) {
        if (lane == 0) {
            atomicCAS(P.status, 0, (int)RSV_ETIMEOUT);
            // let copies still in flight land before the CTA exits (bounded)
            const uint64_t limit = global_timer() + 1000000000ull;
            for (int q = 0; q < NSD + NSE; ++q)
                if (pending & (1u << q))
                    while (!mbar_try_wait(&bars[q], (phase >> q) & 1u) && global_timer() < limit) {
                    }
        }
        __syncwarp();
    }
}

// Factor rows in warp-step order.  One thread per (tile, step, lane).  Block
// values come from `v` (FP64, or the FP32 copy for mixed precision); D^{-1}
// from the FP64 factor; both are stored as T.
template <typename T, typename Tv>
__global__ void pack_tiles(const TileSys *__restrict__ tsys, const int *__restrict__ tile_sys,
                           const int64_t *__restrict__ tile_row0, const int2 *__restrict__ order,
                           const int32_t *__restrict__ rp, const Tv *__restrict__ v,
                           const double *__restrict__ dinv, T *__restrict__ Ff, T *__restrict__ Fb) {
    constexpr int NQP = Bits<T>::NQP;
    const int t = blockIdx.y;
    const TileSys G = tsys[tile_sys[t]];
    const int nx = G.nx, ny = G.ny, nz = G.nz, S = G.S;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= (int64_t)S * 32) return;
    const int lane = (int)(gid & 31);
    const int s = (int)(gid >> 5);
    const int a = lane & 7, b = lane >> 3;
    const int2 JK = order[t];
    const int j = JK.x * TJ + a, k = JK.y * TK + b;
    for (int dir = 0; dir < 2; ++dir) {
        const bool fwd = dir == 0;
        const int i = fwd ? (s - a - b) : (nx - 1 - (s - (TJ - 1 - a) - (TK - 1 - b)));
        T *out = (fwd ? Ff : Fb) + (((size_t)tile_row0[t] + s) * 32 + lane) * NQP;
        const bool valid = j < ny && k < nz && i >= 0 && i < nx;
        for (int q = 0; q < NQP; ++q) out[q] = T(0);
        if (!valid) continue;
        const int64_t c = G.cell0 + (int64_t)k * nx * ny + (int64_t)j * nx + i;
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
            if (sl[blk] >= 0)
                for (int e = 0; e < 9; ++e) out[blk * 9 + e] = (T)v[9 * ((int64_t)rp[c] + sl[blk]) + e];
        for (int e = 0; e < 9; ++e) out[27 + e] = (T)dinv[9 * c + e];
    }
}

// Before a forward sweep: r into tile order, and the forward edge buffers to
// the sentinel.  One thread per (tile, step, lane).
template <typename T>
__global__ void gather_tiles(const TileSys *__restrict__ tsys, const int *__restrict__ tile_sys,
                             const int64_t *__restrict__ tile_row0, const int2 *__restrict__ order,
                             const T *__restrict__ r, T *__restrict__ Vt, T *__restrict__ EJ, T *__restrict__ EK) {
    using U = typename Bits<T>::U;
    const int t = blockIdx.y;
    const TileSys G = tsys[tile_sys[t]];
    const int nx = G.nx, ny = G.ny, nz = G.nz, S = G.S;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= (int64_t)S * 32) return;
    const int lane = (int)(gid & 31);
    const int s = (int)(gid >> 5);
    const int a = lane & 7, b = lane >> 3;
    const int2 JK = order[t];
    const int j = JK.x * TJ + a, k = JK.y * TK + b, i = s - a - b;
    const size_t row = (size_t)tile_row0[t] + s;
    T *o = Vt + (row * 32 + lane) * 4;
    if (j < ny && k < nz && i >= 0 && i < nx) {
        const int64_t c = G.cell0 + (int64_t)k * nx * ny + (int64_t)j * nx + i;
        o[0] = r[3 * c];
        o[1] = r[3 * c + 1];
        o[2] = r[3 * c + 2];
    } else {
        o[0] = o[1] = o[2] = T(0);
    }
    o[3] = T(0);
    // edge buffers [row][TK][4] and [row][TJ][4]: the 32 threads of a (t, s) row
    // cover its 16 + 32 entries
    if (lane < TK * 4) reinterpret_cast<U *>(EJ)[row * TK * 4 + lane] = Bits<T>::SENT;
    reinterpret_cast<U *>(EK)[row * TJ * 4 + lane] = Bits<T>::SENT;
}

}  // namespace

template <typename T>
cudaError_t tiles_setup(const rsv_mat *A, const double *dinv, IluTiles *Tl) {
    using St = Stage<T>;
    cudaError_t e = cudaSuccess;
    if (!Tl->Ff || Tl->elem != (int)sizeof(T)) {
        free_tiles(Tl);
        // tiles of every grid, each grid's tiles in order of J+K, grids one after another
        std::vector<TileSys> sys;
        std::vector<int2> order;
        std::vector<int> tile_sys, pos;
        std::vector<int64_t> row0;
        int64_t rows = 0;
        int maxS = 0;
        for (int g = 0; g < A->nsys; ++g) {
            const SysGrid &sg = A->h_sys[g];
            TileSys ts;
            ts.nx = sg.nx;
            ts.ny = sg.ny;
            ts.nz = sg.nz;
            ts.nTJ = (sg.ny + TJ - 1) / TJ;
            ts.nTK = (sg.nz + TK - 1) / TK;
            ts.S = sg.nx + TJ + TK - 2;
            ts.cell0 = sg.cell0;
            ts.poff = (int)order.size();
            maxS = std::max(maxS, ts.S);
            pos.resize(order.size() + (size_t)ts.nTJ * ts.nTK);
            for (int d = 0; d <= ts.nTJ + ts.nTK - 2; ++d)
                for (int J = 0; J < ts.nTJ; ++J) {
                    const int K = d - J;
                    if (K < 0 || K >= ts.nTK) continue;
                    pos[ts.poff + J * ts.nTK + K] = (int)order.size();
                    order.push_back(make_int2(J, K));
                    tile_sys.push_back(g);
                    row0.push_back(rows);
                    rows += ts.S;
                }
            sys.push_back(ts);
        }
        const int nT = (int)order.size();
        if (nT > 65535) return cudaErrorInvalidConfiguration;  // tiles index blockIdx.y of the pack/gather grids
        Tl->nT = nT;
        Tl->maxS = maxS;
        Tl->rows = rows;
        Tl->elem = (int)sizeof(T);
        auto alloc = [&](void **p, size_t bytes) {
            if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        };
        alloc(&Tl->Ff, rows * St::FB);
        alloc(&Tl->Fb, rows * St::FB);
        alloc(&Tl->Vf, rows * St::VB);
        alloc(&Tl->Vb, rows * St::VB);
        alloc(&Tl->EJf, rows * St::EJB);
        alloc(&Tl->EKf, rows * St::EKB);
        alloc(&Tl->EJb, rows * St::EJB);
        alloc(&Tl->EKb, rows * St::EKB);
        alloc((void **)&Tl->order, sizeof(int2) * nT);
        alloc((void **)&Tl->pos_of, sizeof(int) * nT);
        alloc((void **)&Tl->tile_sys, sizeof(int) * nT);
        alloc((void **)&Tl->tile_row0, sizeof(int64_t) * nT);
        alloc((void **)&Tl->tsys, sizeof(TileSys) * sys.size());
        if (e != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(Tl->order, order.data(), sizeof(int2) * nT, cudaMemcpyHostToDevice, A->stream)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(Tl->pos_of, pos.data(), sizeof(int) * nT, cudaMemcpyHostToDevice, A->stream)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(Tl->tile_sys, tile_sys.data(), sizeof(int) * nT, cudaMemcpyHostToDevice,
                                 A->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(Tl->tile_row0, row0.data(), sizeof(int64_t) * nT, cudaMemcpyHostToDevice,
                                 A->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(Tl->tsys, sys.data(), sizeof(TileSys) * sys.size(), cudaMemcpyHostToDevice,
                                 A->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(A->stream)) != cudaSuccess)
            return e;
        int dev = 0, sms = 0, per_f = 0, per_b = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t smem = (Bits<T>::NSD * St::SIZE + NSE * St::ESIZE) * sizeof(T) +
                            (Bits<T>::NSD + NSE) * sizeof(uint64_t);
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
    const dim3 g((unsigned)((Tl->maxS * 32 + 255) / 256), (unsigned)Tl->nT);
    rsv::count_launches(1);
    if (sizeof(T) == 8)
        pack_tiles<T, double><<<g, 256, 0, A->stream>>>(Tl->tsys, Tl->tile_sys, Tl->tile_row0, Tl->order, A->d_rp,
                                                        A->d_v, dinv, (T *)Tl->Ff, (T *)Tl->Fb);
    else
        pack_tiles<T, float><<<g, 256, 0, A->stream>>>(Tl->tsys, Tl->tile_sys, Tl->tile_row0, Tl->order, A->d_rp,
                                                       A->d_v32, dinv, (T *)Tl->Ff, (T *)Tl->Fb);
    return cudaGetLastError();
}

void free_tiles(IluTiles *Tl) {
    for (void *p : {Tl->Ff, Tl->Fb, Tl->Vf, Tl->Vb, Tl->EJf, Tl->EKf, Tl->EJb, Tl->EKb, (void *)Tl->order,
                    (void *)Tl->pos_of, (void *)Tl->tile_sys, (void *)Tl->tile_row0, (void *)Tl->tsys})
        if (p) cudaFree(p);
    *Tl = IluTiles();
}

template <typename T>
cudaError_t launch_ilu_apply_tiles(const rsv_mat *A, const IluTiles &Tl, const T *r, T *z, const int *done,
                                   int *status, unsigned long long timeout_ns) {
    rsv::count_launches(3);
    const dim3 g((unsigned)((Tl.maxS * 32 + 255) / 256), (unsigned)Tl.nT);
    gather_tiles<T><<<g, 256, 0, A->stream>>>(Tl.tsys, Tl.tile_sys, Tl.tile_row0, Tl.order, r, (T *)Tl.Vf,
                                              (T *)Tl.EJf, (T *)Tl.EKf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SweepArgs<T> f{Tl.nT, Tl.tsys, Tl.tile_sys, Tl.tile_row0, Tl.order, Tl.pos_of, (const T *)Tl.Ff,
                   (const T *)Tl.Vf, (T *)Tl.Vb, nullptr, (T *)Tl.EJf, (T *)Tl.EKf, (T *)Tl.EJb, (T *)Tl.EKb,
                   done, status, timeout_ns};
    SweepArgs<T> bw{Tl.nT, Tl.tsys, Tl.tile_sys, Tl.tile_row0, Tl.order, Tl.pos_of, (const T *)Tl.Fb,
                    (const T *)Tl.Vb, nullptr, z, (T *)Tl.EJb, (T *)Tl.EKb, nullptr, nullptr,
                    done, status, timeout_ns};
    void *fa[] = {&f};
    void *ba[] = {&bw};
    e = cudaLaunchCooperativeKernel((const void *)ilu_sweep_tiles<T, true>, dim3(Tl.grid), dim3(32), fa, Tl.smem,
                                    A->stream);
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
