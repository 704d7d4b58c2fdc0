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
// TMA bulk copies (cp.async.bulk + mbarrier):
//   * the factor row of each lane (three off-diagonal blocks and D^{-1}, 36
//     values, packed at setup in exactly the order the warp reads them) and
//     the input vector, gathered into the same tile order before the sweep.
//     These come in groups of GS steps (one mbarrier, two copies per group)
//     through a ring of NG groups, so a copy is issued NG - 1 groups ahead;
//   * the values of neighbouring tiles' edge cells, ELA steps ahead.  A tile
//     publishes the results of its last j-row and last k-layer into small
//     per-tile edge buffers indexed by the step at which the neighbour will
//     need them.  The buffers hold a signalling-NaN sentinel until written
//     (arithmetic never produces one), so a consumer that finds the sentinel
//     in its staged copy re-reads the value from global memory until it
//     appears (bounded by a time limit that ends the sweep with
//     RSV_ETIMEOUT).
//
// A step is written for few instructions on its dependency chain: GS steps are
// unrolled so every ring offset is a constant, the lead lane's edge copies are
// predicated instead of branched around (a divergent branch cost waiting tiles
// more than it saved), the sentinel test is one warp vote, and results leave in
// 16-byte stores.
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
// Edge ring: NSE stages, neighbour values copied ELA steps ahead.  Each step of
// look-ahead is a step of lag per tile hand-off on the sweep's critical path, so
// the copies run one step ahead (measured on 100x100x50, FP32 apply: 379 us with
// one step, 406 us with two, 462 us with three; per-lane relaxed register loads
// instead of TMA: 595 us).  The stage a step refills (NSE stages: 4 for FP32, 3 for
// FP64) was last read NSE - 1 steps earlier, and its values fed that step's
// results, so those reads are complete and the refill needs no proxy fence (a
// fence there waits for the warp's outstanding stores: 5% slower with it).
constexpr int ELA = 1;
// Steps per data group, GS (Bits<T>).  A tile's step count is padded to a multiple
// of GS (the padded steps hold no valid cell), so every group is full and, GS
// being a multiple of NSE, every edge stage is a constant of the unrolled step.
// FP64 takes three steps per group: 64.5 KB per tile, 3 tiles per SM instead of 2
// (FP64 CPR solve on 256x256x128: 8.71 s against 9.58 s).  FP32 keeps four: three
// would fit 7 tiles per SM instead of 5, but the apply on 256x256x128 then took
// 1.081 ms against 1.061 ms (the wavefront, not residency, bounds it).

template <typename T> struct Bits;
template <> struct Bits<double> {
    using U = unsigned long long;
    static constexpr U SENT = 0xFFF4C0DE5A17E7A1ull;  // signalling NaN
    static constexpr int NQP = 38;                    // padded factor row: conflict-free 16-byte reads
    static constexpr int NG = 2;                      // data ring groups (copies one group ahead)
    static constexpr int GS = 3, NSE = 3;             // steps per data group, edge stages
};
template <> struct Bits<float> {
    using U = unsigned int;
    static constexpr U SENT = 0x7FA5C0DEu;
    static constexpr int NQP = 36;
    static constexpr int NG = 2;
    static constexpr int GS = 4, NSE = 4;
};

// Data stage of one step: factor [32][NQP] and vector [32][4]; a data group holds
// the factor of its GS steps, then their vectors (two contiguous copies).
// Edge stage: edge j [TK][4] | edge k [TJ][4].
template <typename T> struct Stage {
    static constexpr int F = 32 * Bits<T>::NQP;
    static constexpr int V = 32 * 4;
    static constexpr int EJ = TK * 4;
    static constexpr int EK = TJ * 4;
    static constexpr int GS = Bits<T>::GS, NSE = Bits<T>::NSE;
    static_assert(GS % NSE == 0 && ELA >= 1 && ELA < NSE, "edge stages are fixed per unrolled step");
    static constexpr int GSIZE = GS * (F + V);
    static constexpr int ESIZE = EJ + EK;
    static constexpr unsigned FB = F * sizeof(T), VB = V * sizeof(T), EJB = EJ * sizeof(T), EKB = EK * sizeof(T);
};

template <typename T> constexpr size_t sweep_smem() {
    return (size_t)(Bits<T>::NG * Stage<T>::GSIZE + Bits<T>::NSE * Stage<T>::ESIZE) * sizeof(T) +
           (Bits<T>::NG + Bits<T>::NSE) * sizeof(uint64_t);
}

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
// Edge rows of one step into an edge stage, by the lanes whose `go` is set (the
// lead lane): the byte count, then the j row and/or the k row.  Predicated, so
// the warp takes no branch around it.
__device__ __forceinline__ void edge_issue(unsigned go, unsigned goj, unsigned gok, uint64_t *bar, unsigned bytes,
                                           void *dj, const void *sj, unsigned bj, void *dk, const void *sk,
                                           unsigned bk) {
    asm volatile(
        "{\n .reg .pred p, pj, pk;\n"
        " setp.ne.u32 p, %0, 0;\n setp.ne.u32 pj, %1, 0;\n setp.ne.u32 pk, %2, 0;\n"
        " @p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%3], %4;\n"
        " @pj cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%5], [%6], %7, [%3];\n"
        " @pk cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%8], [%9], %10, [%3];\n}" ::"r"(go),
        "r"(goj), "r"(gok), "r"(smem_u32(bar)), "r"(bytes), "r"(smem_u32(dj)), "l"(sj), "r"(bj), "r"(smem_u32(dk)),
        "l"(sk), "r"(bk)
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
// A cell's three results (and a zero pad) as one 16-byte edge-buffer entry.
__device__ __forceinline__ void st_relaxed3(float *p, const float v[3]) {
    asm volatile("st.relaxed.gpu.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(0.f)
                 : "memory");
}
__device__ __forceinline__ void st_relaxed3(double *p, const double v[3]) {
    asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v[0]), "d"(v[1]) : "memory");
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p + 2), "l"(__double_as_longlong(v[2])) : "memory");
}
__device__ __forceinline__ unsigned long long bits_of(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned bits_of(float v) { return __float_as_uint(v); }
__device__ __forceinline__ double value_of(unsigned long long v) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ float value_of(unsigned v) { return __uint_as_float(v); }
template <typename T> __device__ __forceinline__ bool is_sent3(const T v[3]) {
    return bits_of(v[0]) == Bits<T>::SENT || bits_of(v[1]) == Bits<T>::SENT || bits_of(v[2]) == Bits<T>::SENT;
}
// Three values of a 16-byte-aligned shared-memory entry.
__device__ __forceinline__ void lds3(const float *p, float v[3]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
}
__device__ __forceinline__ void lds3(const double *p, double v[3]) {
    const double2 q = *reinterpret_cast<const double2 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = p[2];
}
// A tile-order vector entry: three values and the pad slot.
__device__ __forceinline__ void lds4(const float *p, float v[3], float &pad) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    pad = q.w;
}
__device__ __forceinline__ void lds4(const double *p, double v[3], double &pad) {
    const double2 q0 = reinterpret_cast<const double2 *>(p)[0], q1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    pad = q1.y;
}
// y entry of the backward sweep's tile order (value, value, value, pad).
__device__ __forceinline__ void st3pad(float *p, const float v[3], float pad) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], pad);
}
__device__ __forceinline__ void st3pad(double *p, const double v[3], double pad) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], pad);
}

template <typename T>
struct SweepArgs {
    int nT;                    // tiles of all grids
    const TileSys *tsys;       // per grid
    const int *tile_sys;       // position -> grid
    const int64_t *tile_row0;  // position -> first step row of the tile in the packed arrays
    const int2 *order;         // position -> tile (J, K) inside its grid
    const int *pos_of;         // grid's poff + J * nTK + K -> position
    const T *F;          // factor rows [nT][Sp][32][NQP]
    const T *V;          // input vector in tile order [nT][Sp][32][4]
    T *Vnext;            // forward: y in backward tile order [nT][Sp][32][4]; backward: null
    T *z;                // backward: output in natural order; forward: null
    T *EJ, *EK;          // edge buffers this sweep publishes [nT][Sp][TK][4], [nT][Sp][TJ][4]
    T *EJnext, *EKnext;  // forward: the backward sweep's edge buffers (reset to the sentinel)
    const int *done;
    int *status;
    unsigned long long timeout_ns;
};

template <typename T, bool FWD>
__global__ void __launch_bounds__(32) ilu_sweep_tiles(SweepArgs<T> P) {
    using St = Stage<T>;
    using U = typename Bits<T>::U;
    constexpr int NQP = Bits<T>::NQP;
    constexpr int NG = Bits<T>::NG;
    constexpr int GS = Bits<T>::GS, NSE = Bits<T>::NSE;
    // (No pdl_trigger here: letting the next kernel's CTAs be scheduled beside the sweep slowed the
    // FP32 apply on 256x256x128 from 1.034 to 1.069 ms.)
    if (P.done && *(volatile const int *)P.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    T *ring = reinterpret_cast<T *>(smem);                                   // NG data groups
    T *ering = ring + NG * St::GSIZE;                                        // NSE edge stages
    uint64_t *bars = reinterpret_cast<uint64_t *>(ering + NSE * St::ESIZE);  // NG data + NSE edge barriers
    uint64_t *ebars = bars + NG;
    const int lane = threadIdx.x;
    const int a = lane & 7, b = lane >> 3;
    const unsigned lead = lane == 0;
    if (lead) {
        for (int q = 0; q < NG + NSE; ++q) mbar_init(&bars[q], 1);
        fence_barrier_init();
    }
    __syncwarp();
    unsigned phase = 0, pending = 0;  // bit q: data group stage q; bit NG + q: edge stage q
    const uint64_t deadline = global_timer() + P.timeout_ns;
    bool failed = false;

    auto wait_bar = [&](uint64_t *bar, int bit) {
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

    for (int t = blockIdx.x; t < P.nT && !failed; t += gridDim.x) {
        const int tt = FWD ? t : (P.nT - 1 - t);
        const TileSys G = P.tsys[P.tile_sys[tt]];
        const int nx = G.nx, ny = G.ny, nz = G.nz, S = G.S, Sp = G.Sp, nTJ = G.nTJ, nTK = G.nTK;
        const int ngr = Sp / GS;
        const int2 JK = P.order[tt];
        // producers of this tile's edge inputs (same grid)
        const int pj = FWD ? (JK.x > 0 ? P.pos_of[G.poff + (JK.x - 1) * nTK + JK.y] : -1)
                           : (JK.x + 1 < nTJ ? P.pos_of[G.poff + (JK.x + 1) * nTK + JK.y] : -1);
        const int pk = FWD ? (JK.y > 0 ? P.pos_of[G.poff + JK.x * nTK + JK.y - 1] : -1)
                           : (JK.y + 1 < nTK ? P.pos_of[G.poff + JK.x * nTK + JK.y + 1] : -1);
        const int j = JK.x * TJ + a, k = JK.y * TK + b;
        const bool jk_ok = (j < ny) && (k < nz);
        // Lanes on the tile's lower j (k) face take that neighbour from the edge stage,
        // which holds zeros where the tile has no producer; inner lanes take it from the
        // adjacent lane, whose previous result is zero where it held no cell.
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
        const bool edges = pj >= 0 || pk >= 0;
        const unsigned edge_bytes = (pj >= 0 ? St::EJB : 0u) + (pk >= 0 ? St::EKB : 0u);
        __syncwarp();  // the previous tile's reads of the rings are done
        if (FWD) {
            // this tile's backward-sweep edge buffers start at the sentinel
            U *ej = reinterpret_cast<U *>(P.EJnext + tile0 * St::EJ);
            U *ek = reinterpret_cast<U *>(P.EKnext + tile0 * St::EK);
            for (int q = lane; q < Sp * St::EJ; q += 32) ej[q] = Bits<T>::SENT;
            for (int q = lane; q < Sp * St::EK; q += 32) ek[q] = Bits<T>::SENT;
        }
        // faces without a producer read zeros from the edge stages (no copy writes them)
        if (pj < 0)
            for (int q = lane; q < NSE * St::EJ; q += 32) ering[(q / St::EJ) * St::ESIZE + q % St::EJ] = T(0);
        if (pk < 0)
            for (int q = lane; q < NSE * St::EK; q += 32) ering[(q / St::EK) * St::ESIZE + St::EJ + q % St::EK] = T(0);
        __syncwarp();
        if (lead) {
            fence_proxy_async();
            for (int q = 0; q < NG - 1 && q < ngr; ++q) {
                T *dst = ring + q * St::GSIZE;
                mbar_expect(&bars[q], GS * (St::FB + St::VB));
                tma_load_1d(dst, Ft + (size_t)q * GS * St::F, GS * St::FB, &bars[q]);
                tma_load_1d(dst + GS * St::F, Vt + (size_t)q * GS * St::V, GS * St::VB, &bars[q]);
                pending |= 1u << q;
            }
            if (edges)
                for (int q = 0; q < ELA && q < Sp; ++q) {
                    T *dst = ering + q * St::ESIZE;
                    mbar_expect(&ebars[q], edge_bytes);
                    if (pj >= 0) tma_load_1d(dst, P.EJ + (rowj + q) * St::EJ, St::EJB, &ebars[q]);
                    if (pk >= 0) tma_load_1d(dst + St::EJ, P.EK + (rowk + q) * St::EK, St::EKB, &ebars[q]);
                    pending |= 1u << (NG + q);
                }
        }
        T prev[3] = {T(0), T(0), T(0)};
        int i = FWD ? -off : (nx - 1 + off);  // this lane's cell along x at the current step
        // Per-group running addresses; a step adds a constant offset to each.
        T *yout = FWD ? P.Vnext + ((tile0 + (S - 1)) * 32 + lane) * 4 : P.z + 3 * (base + i);
        constexpr ptrdiff_t ystep = FWD ? -(ptrdiff_t)(32 * 4) : -3;
        T *pubj = P.EJ + ((ptrdiff_t)tile0 - (TJ - 1)) * St::EJ + b * 4;  // row of step s - (TJ - 1)
        T *pubk = P.EK + ((ptrdiff_t)tile0 - (TK - 1)) * St::EK + a * 4;
        const T *pollj = P.EJ + rowj * St::EJ + b * 4;  // the j producer's row of step s
        const T *pollk = P.EK + rowk * St::EK + a * 4;
        const T *ejsrc = P.EJ + (rowj + ELA) * St::EJ;  // edge rows of step s + ELA
        const T *eksrc = P.EK + (rowk + ELA) * St::EK;
        const unsigned goj = lead && pj >= 0, gok = lead && pk >= 0, go = goj | gok;
        int gst = 0;  // data group stage of the current group

        for (int g = 0; g < ngr; ++g) {
            // refill the stage the previous group used (every lane is past it) with group g + NG - 1
            __syncwarp();
            if (lead && g + NG - 1 < ngr) {
                const int q = gst == 0 ? NG - 1 : gst - 1;
                T *dst = ring + q * St::GSIZE;
                fence_proxy_async();
                mbar_expect(&bars[q], GS * (St::FB + St::VB));
                tma_load_1d(dst, Ft + (size_t)(g + NG - 1) * GS * St::F, GS * St::FB, &bars[q]);
                tma_load_1d(dst + GS * St::F, Vt + (size_t)(g + NG - 1) * GS * St::V, GS * St::VB, &bars[q]);
                pending |= 1u << q;
            }
            wait_bar(&bars[gst], gst);
            const T *grp = ring + gst * St::GSIZE;
            gst = gst + 1 == NG ? 0 : gst + 1;
            const bool last = g + 1 == ngr;
#pragma unroll
            for (int u = 0; u < GS; ++u) {
                // refill the edge stage of step s + ELA - NSE (done) with the edge rows of step s + ELA.
                // (The warp barrier also reconverges the lanes after the sentinel poll: without it
                // the FP32 apply on 256x256x128 took 1.20 ms against 1.06 ms.)
                __syncwarp();
                const int eq = (u + ELA) % NSE;
                const unsigned more = (u + ELA < GS || !last) && edges;
                edge_issue(go & more, goj & more, gok & more, &ebars[eq], edge_bytes, ering + eq * St::ESIZE,
                           ejsrc + u * St::EJ, St::EJB, ering + eq * St::ESIZE + St::EJ, eksrc + u * St::EK, St::EKB);
                if (lead && more) pending |= 1u << (NG + eq);
                const bool valid = jk_ok && (unsigned)i < (unsigned)nx;
                // in-tile neighbours: previous step's results of the adjacent lanes
                T nj[3], nk[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    nj[e] = __shfl_sync(0xffffffffu, prev[e], lane_j);
                    nk[e] = __shfl_sync(0xffffffffu, prev[e], lane_k);
                }
                // factor row and input of this lane
                T f[NQP];
                {
                    const T *row = grp + u * St::F + lane * NQP;
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
                T vin[3], vpad;  // vpad: the pad slot, carried from the forward input to the output
                lds4(grp + GS * St::F + u * St::V + lane * 4, vin, vpad);
                // neighbours from other tiles
                T ej[3] = {T(0), T(0), T(0)}, ek[3] = {T(0), T(0), T(0)};
                if (edges) {
                    wait_bar(&ebars[u % NSE], NG + u % NSE);
                    const T *estg = ering + (u % NSE) * St::ESIZE;
                    lds3(estg + b * 4, ej);
                    lds3(estg + St::EJ + a * 4, ek);
                    const bool bad = valid && ((edge_j && is_sent3(ej)) || (edge_k && is_sent3(ek)));
                    if (__any_sync(0xffffffffu, bad) && bad) {
                        // not yet published when the copy ran: re-read until it appears
                        const T *gj = pollj + u * St::EJ, *gk = pollk + u * St::EK;
                        unsigned spins = 0;
                        for (;;) {
                            const bool mj = edge_j && is_sent3(ej), mk = edge_k && is_sent3(ek);
                            if (!mj && !mk) break;
                            if (mj)
                                for (int e = 0; e < 3; ++e) ej[e] = value_of(ld_relaxed(gj + e));
                            if (mk)
                                for (int e = 0; e < 3; ++e) ek[e] = value_of(ld_relaxed(gk + e));
                            if ((++spins & 63u) == 0 && global_timer() > deadline) {
                                failed = true;
                                break;
                            }
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    nj[e] = edge_j ? ej[e] : nj[e];
                    nk[e] = edge_k ? ek[e] : nk[e];
                }
                // slots: forward [0] -z [1] -y [2] -x ; backward [0] +x [1] +y [2] +z
                const T *x0 = FWD ? nk : prev;
                const T *x2 = FWD ? prev : nk;
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
                    if (FWD) {
                        st3pad(yout + u * ystep, res, vpad);
                    } else {
                        T *zo = yout + u * ystep;
                        zo[0] = res[0] + vpad;
                        zo[1] = res[1];
                        zo[2] = res[2];
                    }
                    if (pub_j) st_relaxed3(pubj + u * St::EJ, res);
                    if (pub_k) st_relaxed3(pubk + u * St::EK, res);
                }
                i += FWD ? 1 : -1;
#pragma unroll
                for (int e = 0; e < 3; ++e) prev[e] = valid ? res[e] : T(0);
            }
            yout += GS * ystep;
            pubj += GS * St::EJ;
            pubk += GS * St::EK;
            pollj += GS * St::EJ;
            pollk += GS * St::EK;
            ejsrc += GS * St::EJ;
            eksrc += GS * St::EK;
            if (__any_sync(0xffffffffu, failed)) {
                failed = true;
                break;
            }
        }
    }
    if (failed) {
        if (lead) {
            atomicCAS(P.status, 0, (int)RSV_ETIMEOUT);
            // let copies still in flight land before the CTA exits (bounded)
            const uint64_t limit = global_timer() + 1000000000ull;
            for (int q = 0; q < NG + NSE; ++q)
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
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= (int64_t)G.Sp * 32) return;
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

// A tile-order vector entry (three values and the pad slot) as 16-byte stores.
__device__ __forceinline__ void st4(float *p, const float v[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double v[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// Before a forward sweep: r into tile order, and the forward edge buffers to
// the sentinel.  One thread per (tile, lane) and kGatherSteps consecutive steps:
// its cells are consecutive along x, and all their loads are issued before the
// stores (one load per thread left the gather latency-bound).  The entry's pad
// slot takes add[c] (or 0): the forward sweep carries it into y's entry and the
// backward sweep adds it to the cell's first output component.
constexpr int kGatherSteps = 4;
template <typename T>
__global__ void gather_tiles(const TileSys *__restrict__ tsys, const int *__restrict__ tile_sys,
                             const int64_t *__restrict__ tile_row0, const int2 *__restrict__ order,
                             const T *__restrict__ r, const T *__restrict__ add, T *__restrict__ Vt,
                             T *__restrict__ EJ, T *__restrict__ EK) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    using U = typename Bits<T>::U;
    const int t = blockIdx.y;
    const TileSys G = tsys[tile_sys[t]];
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = (int)(gid & 31);
    const int s0 = (int)(gid >> 5) * kGatherSteps;
    if (s0 >= G.Sp) return;
    const int a = lane & 7, b = lane >> 3;
    const int2 JK = order[t];
    const int j = JK.x * TJ + a, k = JK.y * TK + b;
    const bool jk_ok = j < ny && k < nz;
    const int64_t pencil = G.cell0 + (int64_t)k * nx * ny + (int64_t)j * nx;
    T v[kGatherSteps][4];
#pragma unroll
    for (int u = 0; u < kGatherSteps; ++u) {
        const int i = s0 + u - a - b;
        v[u][0] = v[u][1] = v[u][2] = v[u][3] = T(0);
        if (jk_ok && s0 + u < G.Sp && i >= 0 && i < nx) {
            const int64_t c = pencil + i;
            v[u][0] = r[3 * c];
            v[u][1] = r[3 * c + 1];
            v[u][2] = r[3 * c + 2];
            if (add) v[u][3] = add[c];
        }
    }
#pragma unroll
    for (int u = 0; u < kGatherSteps; ++u) {
        if (s0 + u >= G.Sp) break;
        const size_t row = (size_t)tile_row0[t] + s0 + u;
        st4(Vt + (row * 32 + lane) * 4, v[u]);
        // edge buffers [row][TK][4] and [row][TJ][4]: the 32 threads of a (t, s) row
        // cover its 16 + 32 entries
        if (lane < TK * 4) reinterpret_cast<U *>(EJ)[row * TK * 4 + lane] = Bits<T>::SENT;
        reinterpret_cast<U *>(EK)[row * TJ * 4 + lane] = Bits<T>::SENT;
    }
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
            ts.Sp = (ts.S + Bits<T>::GS - 1) / Bits<T>::GS * Bits<T>::GS;
            ts.cell0 = sg.cell0;
            ts.poff = (int)order.size();
            maxS = std::max(maxS, ts.Sp);
            pos.resize(order.size() + (size_t)ts.nTJ * ts.nTK);
            for (int d = 0; d <= ts.nTJ + ts.nTK - 2; ++d)
                for (int J = 0; J < ts.nTJ; ++J) {
                    const int K = d - J;
                    if (K < 0 || K >= ts.nTK) continue;
                    pos[ts.poff + J * ts.nTK + K] = (int)order.size();
                    order.push_back(make_int2(J, K));
                    tile_sys.push_back(g);
                    row0.push_back(rows);
                    rows += ts.Sp;
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
        const size_t smem = sweep_smem<T>();
        if ((e = cudaFuncSetAttribute((const void *)ilu_sweep_tiles<T, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute((const void *)ilu_sweep_tiles<T, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute((const void *)ilu_sweep_tiles<T, true>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess ||
            (e = cudaFuncSetAttribute((const void *)ilu_sweep_tiles<T, false>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
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
                                   int *status, unsigned long long timeout_ns, const T *add0) {
    rsv::count_launches(3);
    const int groups = (Tl.maxS + kGatherSteps - 1) / kGatherSteps;
    const dim3 g((unsigned)((groups * 32 + 255) / 256), (unsigned)Tl.nT);
    cudaError_t e = launch_pdl(gather_tiles<T>, g, dim3(256), 0, A->stream, Tl.tsys, Tl.tile_sys, Tl.tile_row0,
                               Tl.order, r, add0, (T *)Tl.Vf, (T *)Tl.EJf, (T *)Tl.EKf);
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
                                                    const int *, int *, unsigned long long, const double *);
template cudaError_t launch_ilu_apply_tiles<float>(const rsv_mat *, const IluTiles &, const float *, float *,
                                                   const int *, int *, unsigned long long, const float *);

}  // namespace rsv
