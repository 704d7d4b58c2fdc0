// BSR SpMV y = alpha A x + beta y for 3x3 blocks (Section "Algebraic
// Operations", first equation).  One CTA owns R consecutive block rows: it
// stages their contiguous run of block values and column indices in shared
// memory with coalesced loads, then one thread per scalar row forms the
// three-term products against x.
#include "common.cuh"

namespace rsv {
namespace {

constexpr int kRows = 64;  // block rows per CTA (7 blocks max per row)

template <typename T, int R>
__global__ void __launch_bounds__(3 * R) spmv_bsr3_staged(int nb, const int32_t *__restrict__ rp,
                                                          const int32_t *__restrict__ ci,
                                                          const T *__restrict__ v, T alpha,
                                                          const T *__restrict__ x, T beta,
                                                          T *__restrict__ y, const int *done) {
    if (done && *(volatile const int *)done) return;
    __shared__ T sv[R * 7 * 9];
    __shared__ int32_t sci[R * 7];
    __shared__ int32_t srp[R + 1];
    const int r0 = blockIdx.x * R;
    const int nr = min(R, nb - r0);
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) srp[t] = rp[r0 + t];
    __syncthreads();
    const int p0 = srp[0];
    const int np = srp[nr] - p0;
    const T *vsrc = v + (int64_t)p0 * 9;
    for (int q = threadIdx.x; q < np * 9; q += blockDim.x) sv[q] = vsrc[q];
    for (int q = threadIdx.x; q < np; q += blockDim.x) sci[q] = ci[p0 + q];
    __syncthreads();
    const int t = threadIdx.x;
    if (t >= nr * 3) return;
    const int rl = t / 3, e = t - 3 * (t / 3);
    T acc = T(0);
    for (int p = srp[rl] - p0; p < srp[rl + 1] - p0; ++p) {
        const T *a = sv + p * 9 + 3 * e;
        const T *xc = x + 3 * (int64_t)sci[p];
        acc += a[0] * xc[0] + a[1] * xc[1] + a[2] * xc[2];
    }
    const int64_t row = 3 * (int64_t)(r0 + rl) + e;
    y[row] = (beta == T(0)) ? alpha * acc : alpha * acc + beta * y[row];
}

__global__ void cast_f64_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

}  // namespace

cudaError_t launch_spmv_f64(const rsv_mat *A, double alpha, const double *x, double beta, double *y,
                            const int *done) {
    if (A->nb == 0) return cudaSuccess;
    int grid = (int)((A->nb + kRows - 1) / kRows);
    rsv::count_launches(1);
    spmv_bsr3_staged<double, kRows><<<grid, 3 * kRows, 0, A->stream>>>((int)A->nb, A->d_rp, A->d_ci, A->d_v,
                                                                        alpha, x, beta, y, done);
    return cudaGetLastError();
}

cudaError_t launch_spmv_f32(const rsv_mat *A, float alpha, const float *x, float beta, float *y,
                            const int *done) {
    if (A->nb == 0) return cudaSuccess;
    int grid = (int)((A->nb + kRows - 1) / kRows);
    rsv::count_launches(1);
    spmv_bsr3_staged<float, kRows><<<grid, 3 * kRows, 0, A->stream>>>((int)A->nb, A->d_rp, A->d_ci, A->d_v32,
                                                                       alpha, x, beta, y, done);
    return cudaGetLastError();
}

cudaError_t launch_cast_f64_f32(cudaStream_t st, int64_t n, const double *a, float *b) {
    if (n == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    rsv::count_launches(1);
    cast_f64_f32<<<grid, 256, 0, st>>>(n, a, b);
    return cudaGetLastError();
}

}  // namespace rsv
