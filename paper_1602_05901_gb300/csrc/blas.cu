// Vector algebra of the Krylov solvers (Section "Algebraic Operations":
// y = a x + b y, <x,y>, ||x||), fused where a solver step allows it.
// Reductions are deterministic: every CTA writes one partial per output, and
// the last CTA to finish (ticket counter) sums the partials in CTA order.
#include "common.cuh"

namespace rsv {
namespace {

constexpr int kGroup = 16;  // basis vectors reduced per pass in the multi-dot

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool is_done(const int *done) { return done && *(volatile const int *)done; }

// Returns true in exactly one CTA: the last one to pass, after every CTA's
// partials are visible.
__device__ __forceinline__ bool last_cta(unsigned *counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    return am_last;
}

__global__ void __launch_bounds__(kRedThreads) mdot_kernel(int64_t n, const double *__restrict__ w,
                                                           const double *__restrict__ V, int64_t ldv, int k,
                                                           double *partial, double *out, unsigned *counter,
                                                           const int *done) {
    if (is_done(done)) return;
    __shared__ double sm[kGroup][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int g0 = 0; g0 < k; g0 += kGroup) {
        double acc[kGroup];
#pragma unroll
        for (int i = 0; i < kGroup; ++i) acc[i] = 0.0;
        const int kg = min(kGroup, k - g0);
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
            const double wr = w[r];
#pragma unroll
            for (int i = 0; i < kGroup; ++i)
                if (i < kg) acc[i] += wr * V[(int64_t)(g0 + i) * ldv + r];
        }
#pragma unroll
        for (int i = 0; i < kGroup; ++i) {
            if (i < kg) {
                double s = warp_sum(acc[i]);
                if (lane == 0) sm[i][warp] = s;
            }
        }
        __syncthreads();
        if (threadIdx.x < kg) {
            double s = 0.0;
            for (int q = 0; q < kRedThreads / 32; ++q) s += sm[threadIdx.x][q];
            partial[(int64_t)(g0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
        }
        __syncthreads();
    }
    if (last_cta(counter)) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&partial[(int64_t)i * gridDim.x + b]);
            out[i] = s;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

__global__ void __launch_bounds__(kRedThreads) maxpy_kernel(int64_t n, const double *base,
                                                            const double *__restrict__ V, int64_t ldv, int k,
                                                            const double *c, double sgn, double *out,
                                                            double *partial, double *nrm, unsigned *counter,
                                                            const int *done) {
    if (is_done(done)) return;
    __shared__ double sc[kMaxRestart + 1];
    __shared__ double sm[kRedThreads / 32];
    for (int i = threadIdx.x; i < k; i += blockDim.x) sc[i] = sgn * c[i];
    __syncthreads();
    double ss = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        double acc = base ? base[r] : 0.0;
        for (int i = 0; i < k; ++i) acc += sc[i] * V[(int64_t)i * ldv + r];
        out[r] = acc;
        ss += acc * acc;
    }
    if (!nrm) return;
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) s += sm[q];
        partial[blockIdx.x] = s;
    }
    if (last_cta(counter)) {
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&partial[b]);
            *nrm = sqrt(s);
            *counter = 0u;
        }
    }
}

__global__ void __launch_bounds__(kRedThreads) dot_kernel(int64_t n, const double *__restrict__ x,
                                                          const double *__restrict__ y, double *partial,
                                                          double *out, unsigned *counter, int sqrt_out,
                                                          const int *done) {
    if (is_done(done)) return;
    __shared__ double sm[kRedThreads / 32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) acc += x[r] * y[r];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) s += sm[q];
        partial[blockIdx.x] = s;
    }
    if (last_cta(counter)) {
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&partial[b]);
            *out = sqrt_out ? sqrt(s) : s;
            *counter = 0u;
        }
    }
}

__global__ void axpby_kernel(int64_t n, double a, const double *x, double b, const double *y, double *z) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride)
        z[r] = (b == 0.0) ? a * x[r] : a * x[r] + b * y[r];
}

__global__ void scale_inv_kernel(int64_t n, double *x, const double *s, const int *done) {
    if (is_done(done)) return;
    const double f = 1.0 / *s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) x[r] *= f;
}

int elementwise_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

cudaError_t launch_mdot(cudaStream_t st, int64_t n, const double *w, const double *V, int64_t ldv, int k,
                        double *partial, double *out, unsigned *counter, const int *done) {
    rsv::count_launches(1);
    mdot_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, w, V, ldv, k, partial, out, counter, done);
    return cudaGetLastError();
}

cudaError_t launch_maxpy(cudaStream_t st, int64_t n, const double *base, const double *V, int64_t ldv, int k,
                         const double *c, double sgn, double *out, double *partial, double *nrm,
                         unsigned *counter, const int *done) {
    rsv::count_launches(1);
    maxpy_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, base, V, ldv, k, c, sgn, out, partial, nrm, counter,
                                                     done);
    return cudaGetLastError();
}

cudaError_t launch_dot(cudaStream_t st, int64_t n, const double *x, const double *y, double *partial,
                       double *out, unsigned *counter, int sqrt_out, const int *done) {
    rsv::count_launches(1);
    dot_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, x, y, partial, out, counter, sqrt_out, done);
    return cudaGetLastError();
}

cudaError_t launch_axpby(cudaStream_t st, int64_t n, double a, const double *x, double b, const double *y,
                         double *z) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    axpby_kernel<<<elementwise_grid(n), 256, 0, st>>>(n, a, x, b, y, z);
    return cudaGetLastError();
}

cudaError_t launch_scale_inv(cudaStream_t st, int64_t n, double *x, const double *s, const int *done) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    scale_inv_kernel<<<elementwise_grid(n), 256, 0, st>>>(n, x, s, done);
    return cudaGetLastError();
}

}  // namespace rsv
