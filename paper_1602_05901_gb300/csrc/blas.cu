// Vector algebra of the Krylov solvers (Section "Algebraic Operations":
// y = a x + b y, <x,y>, ||x||), fused where a solver step allows it.
// Vectors are FP64 or FP32 (the inner solves of mixed precision); every
// reduction accumulates in FP64.  Reductions are deterministic: every CTA
// writes one partial per output, and the last CTA to finish (ticket counter)
// sums the partials in CTA order.
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

// Product of two vector entries, exact in FP64 for FP32 inputs.
template <typename T>
__device__ __forceinline__ double prod(T a, T b) {
    return (double)a * (double)b;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) mdot_kernel(int64_t n, const T *__restrict__ w,
                                                           const T *__restrict__ V, int64_t ldv, int k,
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
            const T wr = w[r];
#pragma unroll
            for (int i = 0; i < kGroup; ++i)
                if (i < kg) acc[i] += prod(wr, V[(int64_t)(g0 + i) * ldv + r]);
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

// out = base + sgn * sum_i c_i V_i, in the vector precision; ||out|| in FP64.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) maxpy_kernel(int64_t n, const T *base, const T *__restrict__ V,
                                                            int64_t ldv, int k, const double *c, double sgn, T *out,
                                                            double *partial, double *nrm, unsigned *counter,
                                                            const int *done) {
    if (is_done(done)) return;
    __shared__ T sc[kMaxRestart + 1];
    __shared__ double sm[kRedThreads / 32];
    for (int i = threadIdx.x; i < k; i += blockDim.x) sc[i] = (T)(sgn * c[i]);
    __syncthreads();
    double ss = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        T acc = base ? base[r] : T(0);
        for (int i = 0; i < k; ++i) acc += sc[i] * V[(int64_t)i * ldv + r];
        out[r] = acc;
        ss += prod(acc, acc);
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

template <typename T>
__global__ void __launch_bounds__(kRedThreads) dot_kernel(int64_t n, const T *__restrict__ x,
                                                          const T *__restrict__ y, double *partial, double *out,
                                                          unsigned *counter, int sqrt_out, const int *done) {
    if (is_done(done)) return;
    __shared__ double sm[kRedThreads / 32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) acc += prod(x[r], y[r]);
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

template <typename T>
__global__ void axpby_kernel(int64_t n, T a, const T *x, T b, const T *y, T *z) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride)
        z[r] = (b == T(0)) ? a * x[r] : a * x[r] + b * y[r];
}

template <typename T>
__global__ void scale_inv_kernel(int64_t n, T *x, const double *s, const int *done) {
    if (is_done(done)) return;
    const T f = (T)(1.0 / *s);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) x[r] *= f;
}

// Mixed-precision glue: xf = (float)(x / *s); x += (*s) * (double)df.
__global__ void to_f32_scaled(int64_t n, const double *__restrict__ x, const double *s, float *__restrict__ xf) {
    const double f = 1.0 / *s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) xf[r] = (float)(x[r] * f);
}

__global__ void add_f32_scaled(int64_t n, const float *__restrict__ df, const double *s, double *__restrict__ x) {
    const double f = *s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) x[r] += f * (double)df[r];
}

int elementwise_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

template <typename T>
cudaError_t launch_mdot(cudaStream_t st, int64_t n, const T *w, const T *V, int64_t ldv, int k, double *partial,
                        double *out, unsigned *counter, const int *done) {
    rsv::count_launches(1);
    mdot_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(n, w, V, ldv, k, partial, out, counter, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_maxpy(cudaStream_t st, int64_t n, const T *base, const T *V, int64_t ldv, int k, const double *c,
                         double sgn, T *out, double *partial, double *nrm, unsigned *counter, const int *done) {
    rsv::count_launches(1);
    maxpy_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(n, base, V, ldv, k, c, sgn, out, partial, nrm, counter, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dot(cudaStream_t st, int64_t n, const T *x, const T *y, double *partial, double *out,
                       unsigned *counter, int sqrt_out, const int *done) {
    rsv::count_launches(1);
    dot_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(n, x, y, partial, out, counter, sqrt_out, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpby(cudaStream_t st, int64_t n, T a, const T *x, T b, const T *y, T *z) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    axpby_kernel<T><<<elementwise_grid(n), 256, 0, st>>>(n, a, x, b, y, z);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_inv(cudaStream_t st, int64_t n, T *x, const double *s, const int *done) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    scale_inv_kernel<T><<<elementwise_grid(n), 256, 0, st>>>(n, x, s, done);
    return cudaGetLastError();
}

cudaError_t launch_to_f32_scaled(cudaStream_t st, int64_t n, const double *x, const double *s, float *xf) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    to_f32_scaled<<<elementwise_grid(n), 256, 0, st>>>(n, x, s, xf);
    return cudaGetLastError();
}

cudaError_t launch_add_f32_scaled(cudaStream_t st, int64_t n, const float *df, const double *s, double *x) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    add_f32_scaled<<<elementwise_grid(n), 256, 0, st>>>(n, df, s, x);
    return cudaGetLastError();
}

#define RSV_BLAS_INST(T)                                                                                            \
    template cudaError_t launch_mdot<T>(cudaStream_t, int64_t, const T *, const T *, int64_t, int, double *,       \
                                        double *, unsigned *, const int *);                                        \
    template cudaError_t launch_maxpy<T>(cudaStream_t, int64_t, const T *, const T *, int64_t, int, const double *, \
                                         double, T *, double *, double *, unsigned *, const int *);                 \
    template cudaError_t launch_dot<T>(cudaStream_t, int64_t, const T *, const T *, double *, double *, unsigned *, \
                                       int, const int *);                                                           \
    template cudaError_t launch_axpby<T>(cudaStream_t, int64_t, T, const T *, T, const T *, T *);                  \
    template cudaError_t launch_scale_inv<T>(cudaStream_t, int64_t, T *, const double *, const int *);
RSV_BLAS_INST(double)
RSV_BLAS_INST(float)

}  // namespace rsv
