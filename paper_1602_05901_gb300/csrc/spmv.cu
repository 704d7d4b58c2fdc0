// BSR SpMV y = alpha A x + beta y for 3x3 blocks (Section "Algebraic
// Operations", first equation).
#include "common.cuh"

namespace rsv {
namespace {

constexpr int kRows = 128;  // block rows per CTA (at most 7 blocks per row)

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The seven-point pattern of a single-grid matrix (grid dims; cells in natural order, a row's
// columns ascending: -z, -y, -x, self, +x, +y, +z, absent faces skipped).  Its column indices
// and row pointers follow from the cell index, so the stage-two residual reads neither array.
// Quotients by nx and ny use Div32 (a multiply and a shift).
struct Grid7 {
    int nx, ny, nz;
    Div32 dx, dy;
    static Grid7 of(int nx, int ny, int nz) { return {nx, ny, nz, Div32::of(nx), Div32::of(ny)}; }
};

// Cell c's coordinates (q: pencils before c's; k: planes before c's).
struct Cell7 {
    int c, i, j, k, q;
    __device__ __forceinline__ Cell7(int c_, const Grid7 &g) : c(c_) {
        q = g.dx(c);
        i = c - q * g.nx;
        k = g.dy(q);
        j = q - k * g.ny;
    }
    // First block of row c: 7 c less the faces absent from the cells before c (x: two per
    // complete pencil, and the -x face of c's pencil start; y: 2 nx per complete plane, then the
    // cells of the current plane on its j = 0 and j = ny - 1 rows; z: the cells before c on the
    // k = 0 and k = nz - 1 planes).
    __device__ __forceinline__ int64_t row_start(const Grid7 &g) const {
        const int64_t nxy = (int64_t)g.nx * g.ny, m = (int64_t)j * g.nx + i;
        const int64_t mx = 2 * (int64_t)q + (i > 0 ? 1 : 0);
        const int64_t my = 2 * (int64_t)g.nx * k + min(m, (int64_t)g.nx) + max((int64_t)0, m - (int64_t)(g.ny - 1) * g.nx);
        const int64_t mz = min((int64_t)c, nxy) + max((int64_t)0, (int64_t)c - (int64_t)(g.nz - 1) * nxy);
        return 7 * (int64_t)c - mx - my - mz;
    }
};

// Shared-memory layout of one CTA: block values | column indices | row pointers | mbarrier.
template <typename T, int R> struct SpmvSmem {
    static constexpr int VALS = R * 7 * 9 + 32 / sizeof(T);  // + room for aligning both ends to 16 bytes
    static constexpr int CI = R * 7 + 8;
    static constexpr size_t BYTES = (size_t)VALS * sizeof(T) + CI * 4 + (R + 4) * 4 + 16;
};

// One CTA owns R consecutive block rows.  Their blocks and column indices are
// contiguous in the BSR arrays, so one thread stages both ranges with two TMA
// bulk copies (aligned down/up to 16 bytes; the arrays carry tail padding)
// while the others load the row pointers; then thread (row, e) forms
// sum_p A_p[e][:] . x[3 col_p : 3 col_p + 3].
template <typename T, int R>
__global__ void __launch_bounds__(3 * R) spmv_bsr3_tma(int nb, const int32_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci, const T *__restrict__ v,
                                                       T alpha, const T *__restrict__ x, T beta, T *__restrict__ y,
                                                       const int *done, int *status, unsigned long long timeout_ns) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (done && *(volatile const int *)done) return;
    using L = SpmvSmem<T, R>;
    extern __shared__ __align__(128) unsigned char smem[];
    T *sv = reinterpret_cast<T *>(smem);
    int32_t *sci = reinterpret_cast<int32_t *>(smem + (size_t)L::VALS * sizeof(T));
    int32_t *srp = sci + L::CI;
    uint64_t *bar = reinterpret_cast<uint64_t *>(srp + R + 4);
    const int r0 = blockIdx.x * R;
    const int nr = min(R, nb - r0);
    const int p0 = rp[r0], p1 = rp[r0 + nr];
    const uintptr_t vb0 = (uintptr_t)(v + (int64_t)p0 * 9), vb1 = (uintptr_t)(v + (int64_t)p1 * 9);
    const uintptr_t va0 = vb0 & ~(uintptr_t)15, va1 = (vb1 + 15) & ~(uintptr_t)15;
    const uintptr_t cb0 = (uintptr_t)(ci + p0), cb1 = (uintptr_t)(ci + p1);
    const uintptr_t ca0 = cb0 & ~(uintptr_t)15, ca1 = (cb1 + 15) & ~(uintptr_t)15;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned bytes = (unsigned)((va1 - va0) + (ca1 - ca0));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sv)),
            "l"(va0), "r"((unsigned)(va1 - va0)), "r"(smem_u32(bar))
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sci)),
            "l"(ca0), "r"((unsigned)(ca1 - ca0)), "r"(smem_u32(bar))
            : "memory");
    }
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) srp[t] = rp[r0 + t] - p0;
    __syncthreads();
    {
        unsigned ok = 0;
        const uint64_t deadline = global_timer() + timeout_ns;
        bool late = false;
        for (;;) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(ok)
                : "r"(smem_u32(bar))
                : "memory");
            if (ok) break;
            // the copy is plain memory traffic; the limit only guards against a stuck wait
            if (global_timer() > deadline) {
                late = true;
                break;
            }
        }
        if (__syncthreads_or(late)) {
            // The staged copies did not arrive in time: record it and write NaN to this CTA's rows, so
            // the output cannot pass for a result; thread 0 then waits (bounded) for the copies still in
            // flight before the CTA releases its shared memory.
            if (threadIdx.x == 0 && status) atomicCAS(status, 0, (int)RSV_ETIMEOUT);
            if (threadIdx.x < 3 * nr) y[3 * (int64_t)r0 + threadIdx.x] = T(__int_as_float(0x7fc00000));
            if (threadIdx.x == 0) {
                const uint64_t drain = global_timer() + 10000000ull;
                do {
                    asm volatile(
                        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, "
                        "0, p;\n}"
                        : "=r"(ok)
                        : "r"(smem_u32(bar))
                        : "memory");
                } while (!ok && global_timer() < drain);
            }
            return;
        }
    }
    const int voff = (int)((vb0 - va0) / sizeof(T));
    const int coff = (int)((cb0 - ca0) / 4);
    const int t = threadIdx.x;
    if (t >= nr * 3) return;
    const int rl = t / 3, e = t - 3 * (t / 3);
    T acc = T(0);
    for (int p = srp[rl]; p < srp[rl + 1]; ++p) {
        const T *a = sv + voff + p * 9 + 3 * e;
        const T *xc = x + 3 * (int64_t)sci[coff + p];
        acc = fma(a[0], xc[0], acc);
        acc = fma(a[1], xc[1], acc);
        acc = fma(a[2], xc[2], acc);
    }
    const int64_t row = 3 * (int64_t)(r0 + rl) + e;
    y[row] = (beta == T(0)) ? alpha * acc : alpha * acc + beta * y[row];
}

// r = f - A (p_c, 0, 0)_c from the pressure columns apc[3 q + e] = A_q[e][0]: the BSR SpMV
// above with one column per block and x = p (CPR-PF's stage-two residual).  Same staging; the
// sum over a row's blocks, and r = -1 * sum + f, round as the full SpMV of (p_c, 0, 0) does.
template <typename T, int R>
__global__ void __launch_bounds__(3 * R) pcol_residual_tma(int nb, const int32_t *__restrict__ rp,
                                                           const int32_t *__restrict__ ci, const T *__restrict__ apc,
                                                           const T *__restrict__ p, const T *__restrict__ f,
                                                           T *__restrict__ r, const int *done, int *status,
                                                           unsigned long long timeout_ns) {
    if (done && *(volatile const int *)done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int VALS = R * 7 * 3 + 32 / sizeof(T);
    constexpr int CI = R * 7 + 8;
    T *sv = reinterpret_cast<T *>(smem);
    int32_t *sci = reinterpret_cast<int32_t *>(smem + (size_t)VALS * sizeof(T));
    int32_t *srp = sci + CI;
    uint64_t *bar = reinterpret_cast<uint64_t *>(srp + R + 4);
    const int r0 = blockIdx.x * R;
    const int nr = min(R, nb - r0);
    const int p0 = rp[r0], p1 = rp[r0 + nr];
    const uintptr_t vb0 = (uintptr_t)(apc + (int64_t)p0 * 3), vb1 = (uintptr_t)(apc + (int64_t)p1 * 3);
    const uintptr_t va0 = vb0 & ~(uintptr_t)15, va1 = (vb1 + 15) & ~(uintptr_t)15;
    const uintptr_t cb0 = (uintptr_t)(ci + p0), cb1 = (uintptr_t)(ci + p1);
    const uintptr_t ca0 = cb0 & ~(uintptr_t)15, ca1 = (cb1 + 15) & ~(uintptr_t)15;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned bytes = (unsigned)((va1 - va0) + (ca1 - ca0));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sv)),
            "l"(va0), "r"((unsigned)(va1 - va0)), "r"(smem_u32(bar))
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sci)),
            "l"(ca0), "r"((unsigned)(ca1 - ca0)), "r"(smem_u32(bar))
            : "memory");
    }
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) srp[t] = rp[r0 + t] - p0;
    const int t = threadIdx.x;
    const int64_t row = 3 * (int64_t)r0 + t;
    const T fr = t < nr * 3 ? f[row] : T(0);  // issued before the wait
    __syncthreads();
    {
        unsigned ok = 0;
        const uint64_t deadline = global_timer() + timeout_ns;
        bool late = false;
        for (;;) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(ok)
                : "r"(smem_u32(bar))
                : "memory");
            if (ok) break;
            if (global_timer() > deadline) {
                late = true;
                break;
            }
        }
        if (__syncthreads_or(late)) {
            if (t == 0 && status) atomicCAS(status, 0, (int)RSV_ETIMEOUT);
            if (t < 3 * nr) r[row] = T(__int_as_float(0x7fc00000));
            if (t == 0) {
                const uint64_t drain = global_timer() + 10000000ull;
                do {
                    asm volatile(
                        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, "
                        "0, p;\n}"
                        : "=r"(ok)
                        : "r"(smem_u32(bar))
                        : "memory");
                } while (!ok && global_timer() < drain);
            }
            return;
        }
    }
    if (t >= nr * 3) return;
    const int voff = (int)((vb0 - va0) / sizeof(T));
    const int coff = (int)((cb0 - ca0) / 4);
    const int rl = t / 3, e = t - 3 * (t / 3);
    T acc = T(0);
    for (int q = srp[rl]; q < srp[rl + 1]; ++q) acc = fma(sv[voff + 3 * q + e], p[sci[coff + q]], acc);
    r[row] = T(-1) * acc + fr;
}

// The stage-two residual on a single-grid seven-point pattern: one thread per block row
// forms its three entries, columns from the cell index, only the pressure columns staged.
// Many small CTAs keep enough copies in flight per SM.  Same sums in the same order as
// pcol_residual_tma.
template <typename T, int R>
__global__ void __launch_bounds__(R) pcol_residual_stencil(int nb, Grid7 g, const T *__restrict__ apc,
                                                           const T *__restrict__ p, const T *__restrict__ f,
                                                           T *__restrict__ r, const int *done, int *status,
                                                           unsigned long long timeout_ns) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (done && *(volatile const int *)done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int VALS = R * 7 * 3 + 32 / sizeof(T);
    T *sv = reinterpret_cast<T *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + ((size_t)VALS * sizeof(T) + 7) / 8 * 8);
    const int r0 = blockIdx.x * R;
    const int nr = min(R, nb - r0);
    const int64_t p0 = Cell7(r0, g).row_start(g), p1 = Cell7(r0 + nr, g).row_start(g);
    const uintptr_t vb0 = (uintptr_t)(apc + p0 * 3), vb1 = (uintptr_t)(apc + p1 * 3);
    const uintptr_t va0 = vb0 & ~(uintptr_t)15, va1 = (vb1 + 15) & ~(uintptr_t)15;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"((unsigned)(va1 - va0))
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sv)),
            "l"(va0), "r"((unsigned)(va1 - va0)), "r"(smem_u32(bar))
            : "memory");
    }
    const int t = threadIdx.x;
    const int64_t row = 3 * (int64_t)(r0 + t);
    T fr[3] = {T(0), T(0), T(0)};
    if (t < nr)  // issued before the wait
        for (int e = 0; e < 3; ++e) fr[e] = f[row + e];
    __syncthreads();
    {
        unsigned ok = 0;
        const uint64_t deadline = global_timer() + timeout_ns;
        bool late = false;
        for (;;) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(ok)
                : "r"(smem_u32(bar))
                : "memory");
            if (ok) break;
            if (global_timer() > deadline) {
                late = true;
                break;
            }
        }
        if (__syncthreads_or(late)) {
            if (t == 0 && status) atomicCAS(status, 0, (int)RSV_ETIMEOUT);
            if (t < nr)
                for (int e = 0; e < 3; ++e) r[row + e] = T(__int_as_float(0x7fc00000));
            if (t == 0) {
                const uint64_t drain = global_timer() + 10000000ull;
                do {
                    asm volatile(
                        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, "
                        "0, p;\n}"
                        : "=r"(ok)
                        : "r"(smem_u32(bar))
                        : "memory");
                } while (!ok && global_timer() < drain);
            }
            return;
        }
    }
    if (t >= nr) return;
    const Cell7 cl(r0 + t, g);
    const T *a = sv + (int)((vb0 - va0) / sizeof(T)) + (int)(cl.row_start(g) - p0) * 3;
    const int64_t c = cl.c, nxy = (int64_t)g.nx * g.ny;
    T acc[3] = {T(0), T(0), T(0)};
    auto blk = [&](int64_t col) {
        const T pc = p[col];
        acc[0] = fma(a[0], pc, acc[0]);
        acc[1] = fma(a[1], pc, acc[1]);
        acc[2] = fma(a[2], pc, acc[2]);
        a += 3;
    };
    if (cl.k > 0) blk(c - nxy);
    if (cl.j > 0) blk(c - g.nx);
    if (cl.i > 0) blk(c - 1);
    blk(c);
    if (cl.i < g.nx - 1) blk(c + 1);
    if (cl.j < g.ny - 1) blk(c + g.nx);
    if (cl.k < g.nz - 1) blk(c + nxy);
    for (int e = 0; e < 3; ++e) r[row + e] = T(-1) * acc[e] + fr[e];
}

__global__ void cast_f64_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

}  // namespace

template <typename T, int R>
cudaError_t spmv_attr() {
    return cudaFuncSetAttribute((const void *)spmv_bsr3_tma<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SpmvSmem<T, R>::BYTES);
}

// The index-free form of the seven-point pattern (columns and row starts from the cell index)
// reads 10% fewer bytes but measured slower on 256x256x128 (FP64 1.09 against 0.97 ms, FP32
// 0.383 against 0.377 ms): the SpMV keeps the staged column indices.
template <typename T, int R>
cudaError_t spmv_launch(const rsv_mat *A, const T *v, T alpha, const T *x, T beta, T *y, const int *done,
                        int *status, unsigned long long timeout_ns) {
    const int grid = (int)((A->nb + R - 1) / R);
    rsv::count_launches(1);
    return launch_pdl(spmv_bsr3_tma<T, R>, dim3(grid), dim3(3 * R), SpmvSmem<T, R>::BYTES, A->stream, (int)A->nb,
                      A->d_rp, A->d_ci, v, alpha, x, beta, y, done, status, timeout_ns);
}

// Block rows per CTA: 32, 64 or 128, picked per matrix and precision by timing (spmv_autotune).
template <typename T>
cudaError_t spmv_dispatch(const rsv_mat *A, const T *v, T alpha, const T *x, T beta, T *y, const int *done,
                          int *status, unsigned long long timeout_ns) {
    if (A->nb == 0) return cudaSuccess;
    switch (sizeof(T) == 8 ? A->spmv_rows64 : A->spmv_rows32) {
    case 32: return spmv_launch<T, 32>(A, v, alpha, x, beta, y, done, status, timeout_ns);
    case 64: return spmv_launch<T, 64>(A, v, alpha, x, beta, y, done, status, timeout_ns);
    default: return spmv_launch<T, kRows>(A, v, alpha, x, beta, y, done, status, timeout_ns);
    }
}

template <typename T, int R> constexpr size_t pcol_smem() {
    return (size_t)(R * 7 * 3 + 32 / sizeof(T)) * sizeof(T) + (R * 7 + 8) * 4 + (R + 4) * 4 + 16;
}
template <typename T, int R> constexpr size_t pcol_stencil_smem() {
    return ((size_t)(R * 7 * 3 + 32 / sizeof(T)) * sizeof(T) + 7) / 8 * 8 + 16;
}

template <typename T>
cudaError_t launch_pressure_residual(const rsv_mat *A, const T *apc, const T *p, const T *f, T *r, const int *done,
                                     int *status, unsigned long long timeout_ns) {
    if (A->nb == 0) return cudaSuccess;
    constexpr int R = 128;
    const int grid = (int)((A->nb + R - 1) / R);
    rsv::count_launches(1);
    if (A->nsys == 1)  // 0.15 ms less per FP32 CPR apply on 256x256x128 than the indexed form
        return launch_pdl(pcol_residual_stencil<T, R>, dim3(grid), dim3(R), pcol_stencil_smem<T, R>(), A->stream,
                          (int)A->nb, Grid7::of(A->nx, A->ny, A->nz), apc, p, f, r, done, status, timeout_ns);
    else
        pcol_residual_tma<T, R><<<grid, 3 * R, pcol_smem<T, R>(), A->stream>>>((int)A->nb, A->d_rp, A->d_ci, apc, p,
                                                                              f, r, done, status, timeout_ns);
    return cudaGetLastError();
}
template cudaError_t launch_pressure_residual<double>(const rsv_mat *, const double *, const double *, const double *,
                                                      double *, const int *, int *, unsigned long long);
template cudaError_t launch_pressure_residual<float>(const rsv_mat *, const float *, const float *, const float *,
                                                     float *, const int *, int *, unsigned long long);

cudaError_t spmv_init() {
    cudaError_t e;
    if ((e = spmv_attr<double, 32>()) != cudaSuccess || (e = spmv_attr<double, 64>()) != cudaSuccess ||
        (e = spmv_attr<double, kRows>()) != cudaSuccess || (e = spmv_attr<float, 32>()) != cudaSuccess ||
        (e = spmv_attr<float, 64>()) != cudaSuccess || (e = spmv_attr<float, kRows>()) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute((const void *)pcol_residual_tma<double, 128>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pcol_smem<double, 128>())) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute((const void *)pcol_residual_tma<float, 128>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pcol_smem<float, 128>())) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute((const void *)pcol_residual_stencil<double, 128>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pcol_stencil_smem<double, 128>())) != cudaSuccess ||
        (e = cudaFuncSetAttribute((const void *)pcol_residual_stencil<float, 128>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pcol_stencil_smem<float, 128>())) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t launch_spmv_f64(const rsv_mat *A, double alpha, const double *x, double beta, double *y,
                            const int *done, int *status, unsigned long long timeout_ns) {
    return spmv_dispatch<double>(A, A->d_v, alpha, x, beta, y, done, status, timeout_ns);
}

cudaError_t launch_spmv_f32(const rsv_mat *A, float alpha, const float *x, float beta, float *y,
                            const int *done, int *status, unsigned long long timeout_ns) {
    return spmv_dispatch<float>(A, A->d_v32, alpha, x, beta, y, done, status, timeout_ns);
}

cudaError_t spmv_autotune(rsv_mat *A) {
    if (A->spmv_tuned || A->nb == 0) return cudaSuccess;
    cudaStream_t st = A->stream;
    const int cands[3] = {32, 64, 128};
    double *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&x, sizeof(double) * 3 * A->nb, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&y, sizeof(double) * 3 * A->nb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(double) * 3 * A->nb, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int prec = 0; prec < 2 && e == cudaSuccess; ++prec) {
        if (prec == 1 && !A->d_v32) break;
        int &rows = prec == 0 ? A->spmv_rows64 : A->spmv_rows32;
        float best = 1e30f;
        int pick = rows;
        for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
            rows = cands[q];
            auto run = [&]() {
                return prec == 0 ? launch_spmv_f64(A, 1.0, x, 0.0, y, nullptr)
                                 : launch_spmv_f32(A, 1.0f, (const float *)x, 0.0f, (float *)y, nullptr);
            };
            for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = run();
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            for (int w = 0; w < 5 && e == cudaSuccess; ++w) e = run();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                pick = cands[q];
            }
        }
        rows = pick;
    }
    if (x) cudaFreeAsync(x, st);
    if (y) cudaFreeAsync(y, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) A->spmv_tuned = true;
    return e;
}

cudaError_t launch_cast_f64_f32(cudaStream_t st, int64_t n, const double *a, float *b) {
    if (n == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    rsv::count_launches(1);
    cast_f64_f32<<<grid, 256, 0, st>>>(n, a, b);
    return cudaGetLastError();
}

}  // namespace rsv
