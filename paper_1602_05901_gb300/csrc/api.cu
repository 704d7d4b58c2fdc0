// C ABI of librsv, part 1: status strings, parameter defaults, the grid and
// matrix handles (Sections "Grid", "Distributed Matrices") and the vector
// algebra entry points (Section "Algebraic Operations").  The solver handle
// and the Krylov drivers live in solve.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace rsv {

static thread_local cudaError_t g_last_cuda = cudaSuccess;
static std::atomic<uint64_t> g_launches{0};
void set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

rsv_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RSV_OK;
    set_last_cuda_error(e);
    return (e == cudaErrorMemoryAllocation) ? RSV_ENOMEM : RSV_ECUDA;
}

}  // namespace rsv

using namespace rsv;

extern "C" {

void rsv_solver_params_default(rsv_solver_params *p) {
    if (!p) return;
    p->solver = RSV_GMRES;
    p->restart = 30;
    p->rtol = 1e-8;
    p->atol = 0.0;
    p->btol = 1e-30;
    p->maxit = 2000;
    p->precision = RSV_PREC_FP64;
    p->inner_rtol = 1e-5;
    p->max_outer = 10;
    p->watchdog = 2000000;  // microseconds
}

void rsv_pc_params_default(rsv_pc_params *p) {
    if (!p) return;
    p->gmg_max_levels = 6;
    p->gmg_max_coarse = 512;
    p->gmg_sweeps = 2;
    p->decoupling = 0;
    p->coarsening = 0;
}

const char *rsv_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }

uint64_t rsv_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char *rsv_status_string(rsv_status s) {
    switch (s) {
    case RSV_OK: return "ok";
    case RSV_EINVAL: return "invalid argument";
    case RSV_ENOMEM: return "out of memory";
    case RSV_ECUDA: return "CUDA runtime error";
    case RSV_ENOTSUP: return "not supported";
    case RSV_ESINGULAR: return "singular pivot";
    case RSV_EBREAKDOWN: return "Krylov breakdown";
    case RSV_ENOCONV: return "not converged within maxit";
    case RSV_ETIMEOUT: return "device wait timed out";
    case RSV_ENAN: return "NaN or Inf in a norm";
    }
    return "unknown status";
}

// ------------------------------------------------------------------- grid

rsv_status rsv_grid_create(int nx, int ny, int nz, rsv_grid **out) {
    if (!out || nx < 1 || ny < 1 || nz < 1) return RSV_EINVAL;
    const int64_t nb = (int64_t)nx * ny * nz;
    if (3 * nb >= (1ll << 31) || 7 * nb >= (1ll << 31)) return RSV_EINVAL;
    rsv_grid *g = new (std::nothrow) rsv_grid{nx, ny, nz};
    if (!g) return RSV_ENOMEM;
    *out = g;
    return RSV_OK;
}

void rsv_grid_destroy(rsv_grid *g) { delete g; }

// ----------------------------------------------------------------- matrix

static void mat_free(rsv_mat *A) {
    if (!A) return;
    if (A->d_sys) cudaFree(A->d_sys);
    if (A->d_sys_of_cell) cudaFree(A->d_sys_of_cell);
    if (A->d_rp) cudaFree(A->d_rp);
    if (A->d_ci) cudaFree(A->d_ci);
    if (A->d_v) cudaFree(A->d_v);
    if (A->d_v32) cudaFree(A->d_v32);
    delete A;
}

}  // extern "C"

namespace rsv {

// Seven-point BSR pattern of one grid or of a block-diagonal batch of grids
// (each grid's cells contiguous, bottom-up within the grid).
rsv_status mat_create_grids(const std::vector<int> &dims, cudaStream_t stream, rsv_mat **out, bool with_f32) {
    const int nsys = (int)dims.size() / 3;
    int64_t total = 0;
    for (int s = 0; s < nsys; ++s) {
        if (dims[3 * s] < 1 || dims[3 * s + 1] < 1 || dims[3 * s + 2] < 1) return RSV_EINVAL;
        total += (int64_t)dims[3 * s] * dims[3 * s + 1] * dims[3 * s + 2];
    }
    if (nsys < 1 || 3 * total >= (1ll << 31) || 7 * total >= (1ll << 31)) return RSV_EINVAL;
    rsv_mat *A = new (std::nothrow) rsv_mat();
    if (!A) return RSV_ENOMEM;
    A->nx = dims[0];
    A->ny = dims[1];
    A->nz = dims[2];
    A->nsys = nsys;
    A->nb = total;
    A->stream = stream;
    A->h_rp.resize(A->nb + 1);
    A->h_ci.reserve(7 * A->nb);
    A->h_rp[0] = 0;
    std::vector<int32_t> sys_of_cell(A->nb);
    int64_t c0 = 0;
    for (int s = 0; s < nsys; ++s) {
        const int nx = dims[3 * s], ny = dims[3 * s + 1], nz = dims[3 * s + 2];
        A->h_sys.push_back(SysGrid{nx, ny, nz, 0, c0});
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const int32_t c = (int32_t)(c0 + (int64_t)nx * ny * k + (int64_t)nx * j + i);
                    if (k > 0) A->h_ci.push_back(c - nx * ny);
                    if (j > 0) A->h_ci.push_back(c - nx);
                    if (i > 0) A->h_ci.push_back(c - 1);
                    A->h_ci.push_back(c);
                    if (i < nx - 1) A->h_ci.push_back(c + 1);
                    if (j < ny - 1) A->h_ci.push_back(c + nx);
                    if (k < nz - 1) A->h_ci.push_back(c + nx * ny);
                    A->h_rp[c + 1] = (int32_t)A->h_ci.size();
                    sys_of_cell[c] = s;
                }
        c0 += (int64_t)nx * ny * nz;
    }
    A->nnzb = (int64_t)A->h_ci.size();
    cudaError_t e;
    const size_t vbytes = sizeof(double) * (9 * (size_t)A->nnzb + 16);
    if ((e = cudaMalloc((void **)&A->d_rp, sizeof(int32_t) * (A->nb + 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&A->d_ci, sizeof(int32_t) * (A->nnzb + 16))) != cudaSuccess ||
        (e = cudaMalloc((void **)&A->d_v, vbytes)) != cudaSuccess ||
        (with_f32 && (e = cudaMalloc((void **)&A->d_v32, vbytes / 2)) != cudaSuccess) ||
        (e = cudaMalloc((void **)&A->d_sys, sizeof(SysGrid) * nsys)) != cudaSuccess ||
        (e = cudaMalloc((void **)&A->d_sys_of_cell, sizeof(int32_t) * A->nb)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A->d_rp, A->h_rp.data(), sizeof(int32_t) * (A->nb + 1), cudaMemcpyHostToDevice,
                             A->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A->d_ci, A->h_ci.data(), sizeof(int32_t) * A->nnzb, cudaMemcpyHostToDevice,
                             A->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A->d_sys, A->h_sys.data(), sizeof(SysGrid) * nsys, cudaMemcpyHostToDevice,
                             A->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A->d_sys_of_cell, sys_of_cell.data(), sizeof(int32_t) * A->nb, cudaMemcpyHostToDevice,
                             A->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(A->d_ci + A->nnzb, 0, sizeof(int32_t) * 16, A->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(A->d_v, 0, vbytes, A->stream)) != cudaSuccess ||
        (e = spmv_init()) != cudaSuccess ||
        (with_f32 && (e = cudaMemsetAsync(A->d_v32, 0, vbytes / 2, A->stream)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(A->stream)) != cudaSuccess) {
        mat_free(A);
        return cuda_status(e);
    }
    *out = A;
    return RSV_OK;
}

}  // namespace rsv

extern "C" {

rsv_status rsv_mat_create(const rsv_grid *g, void *stream, rsv_mat **out) {
    return rsv_mat_create_bsr(g, 3, RSV_PREC_MIXED, stream, out);
}

rsv_status rsv_mat_create_bsr(const rsv_grid *g, int block, int prec, void *stream, rsv_mat **out) {
    if (!g || !out) return RSV_EINVAL;
    if (prec != RSV_PREC_FP64 && prec != RSV_PREC_MIXED) return RSV_EINVAL;
    if (block != 3) return RSV_ENOTSUP;
    return mat_create_grids({g->nx, g->ny, g->nz}, (cudaStream_t)stream, out, prec == RSV_PREC_MIXED);
}

rsv_status rsv_mat_create_batch(int nsys, const int *dims, void *stream, rsv_mat **out) {
    if (nsys < 1 || nsys > (1 << 20) || !dims || !out) return RSV_EINVAL;
    return mat_create_grids(std::vector<int>(dims, dims + 3 * (size_t)nsys), (cudaStream_t)stream, out, true);
}

rsv_status rsv_mat_get_batch(const rsv_mat *A, int *nsys, int64_t *cell_offsets) {
    if (!A) return RSV_EINVAL;
    if (nsys) *nsys = A->nsys;
    if (cell_offsets) {
        for (int s = 0; s < A->nsys; ++s) cell_offsets[s] = A->h_sys[s].cell0;
        cell_offsets[A->nsys] = A->nb;
    }
    return RSV_OK;
}

void rsv_mat_destroy(rsv_mat *A) {
    if (A) cudaStreamSynchronize(A->stream);
    mat_free(A);
}

rsv_status rsv_mat_get_pattern(const rsv_mat *A, const int32_t **row_ptr, const int32_t **col_idx, int64_t *nb,
                               int64_t *nnzb) {
    if (!A) return RSV_EINVAL;
    if (row_ptr) *row_ptr = A->h_rp.data();
    if (col_idx) *col_idx = A->h_ci.data();
    if (nb) *nb = A->nb;
    if (nnzb) *nnzb = A->nnzb;
    return RSV_OK;
}

rsv_status rsv_mat_set_values(rsv_mat *A, const double *vals, int on_device) {
    if (!A || !vals) return RSV_EINVAL;
    const size_t bytes = sizeof(double) * 9 * (size_t)A->nnzb;
    RSV_CUDA_TRY(cudaMemcpyAsync(A->d_v, vals, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 A->stream));
    if (A->d_v32) RSV_CUDA_TRY(launch_cast_f64_f32(A->stream, 9 * A->nnzb, A->d_v, A->d_v32));
    RSV_CUDA_TRY(spmv_autotune(A));  // first values only: time the SpMV tile candidates on this pattern
    if (!on_device) RSV_CUDA_TRY(cudaStreamSynchronize(A->stream));
    A->version++;
    return RSV_OK;
}

rsv_status rsv_spmv(const rsv_mat *A, double alpha, const double *x, double beta, double *y) {
    if (!A || !x || !y) return RSV_EINVAL;
    RSV_CUDA_TRY(launch_spmv_f64(A, alpha, x, beta, y, nullptr));
    return RSV_OK;
}

rsv_status rsv_spmv_f32(const rsv_mat *A, float alpha, const float *x, float beta, float *y) {
    if (!A || !x || !y || !A->d_v32) return RSV_EINVAL;
    RSV_CUDA_TRY(launch_spmv_f32(A, alpha, x, beta, y, nullptr));
    return RSV_OK;
}

// ------------------------------------------------------------------ vectors

}  // extern "C"

namespace rsv {
namespace {

__global__ void cast_f32_f64_kernel(int64_t n, const float *__restrict__ a, double *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

cudaError_t launch_cast_f32_f64(cudaStream_t st, int64_t n, const float *a, double *b) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    cast_f32_f64_kernel<<<(unsigned)std::min<int64_t>(want, 152 * 16), 256, 0, st>>>(n, a, b);
    count_launches(1);
    return cudaGetLastError();
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t elem_bytes(int prec) { return prec == RSV_PREC_FP64 ? sizeof(double) : sizeof(float); }

}  // namespace
}  // namespace rsv

extern "C" {

rsv_status rsv_vec_create(const rsv_grid *g, int prec, void *stream, rsv_vec **out) {
    if (!g || !out || (prec != RSV_PREC_FP64 && prec != RSV_PREC_MIXED)) return RSV_EINVAL;
    rsv_vec *v = new (std::nothrow) rsv_vec();
    if (!v) return RSV_ENOMEM;
    v->n = 3 * (int64_t)g->nx * g->ny * g->nz;
    v->prec = prec;
    v->owned = true;
    cudaError_t e = cudaMalloc(&v->data, std::max<size_t>(16, v->n * elem_bytes(prec)));
    if (e == cudaSuccess) e = cudaMemsetAsync(v->data, 0, v->n * elem_bytes(prec), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        if (v->data) cudaFree(v->data);
        delete v;
        return cuda_status(e);
    }
    *out = v;
    return RSV_OK;
}

rsv_status rsv_vec_wrap(void *dev_ptr, int64_t n, int prec, rsv_vec **out) {
    if (!out || n < 0 || (prec != RSV_PREC_FP64 && prec != RSV_PREC_MIXED)) return RSV_EINVAL;
    if (n > 0 && (!dev_ptr || !is_device_pointer(dev_ptr))) return RSV_EINVAL;
    if ((uintptr_t)dev_ptr % elem_bytes(prec)) return RSV_EINVAL;
    rsv_vec *v = new (std::nothrow) rsv_vec();
    if (!v) return RSV_ENOMEM;
    v->data = dev_ptr;
    v->n = n;
    v->prec = prec;
    v->owned = false;
    *out = v;
    return RSV_OK;
}

void rsv_vec_destroy(rsv_vec *v) {
    if (!v) return;
    if (v->owned && v->data) cudaFree(v->data);  // cudaFree waits for the device's work in flight
    delete v;
}

rsv_status rsv_vec_info(const rsv_vec *v, void **dev_ptr, int64_t *n, int *prec) {
    if (!v) return RSV_EINVAL;
    if (dev_ptr) *dev_ptr = v->data;
    if (n) *n = v->n;
    if (prec) *prec = v->prec;
    return RSV_OK;
}

rsv_status rsv_vec_set(rsv_vec *v, const double *src, int on_device, void *stream) {
    if (!v || (v->n > 0 && !src)) return RSV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (v->n == 0) return RSV_OK;
    if (v->prec == RSV_PREC_FP64) {
        RSV_CUDA_TRY(cudaMemcpyAsync(v->data, src, sizeof(double) * v->n,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        if (!on_device) RSV_CUDA_TRY(cudaStreamSynchronize(st));
        return RSV_OK;
    }
    if (on_device) {
        RSV_CUDA_TRY(launch_cast_f64_f32(st, v->n, src, (float *)v->data));
        return RSV_OK;
    }
    std::vector<float> tmp;
    try {
        tmp.resize(v->n);
    } catch (...) {
        return RSV_ENOMEM;
    }
    for (int64_t i = 0; i < v->n; ++i) tmp[i] = (float)src[i];
    RSV_CUDA_TRY(cudaMemcpyAsync(v->data, tmp.data(), sizeof(float) * v->n, cudaMemcpyHostToDevice, st));
    RSV_CUDA_TRY(cudaStreamSynchronize(st));
    return RSV_OK;
}

rsv_status rsv_vec_get(const rsv_vec *v, double *dst, int on_device, void *stream) {
    if (!v || (v->n > 0 && !dst)) return RSV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (v->n == 0) return RSV_OK;
    if (v->prec == RSV_PREC_FP64) {
        RSV_CUDA_TRY(cudaMemcpyAsync(dst, v->data, sizeof(double) * v->n,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        if (!on_device) RSV_CUDA_TRY(cudaStreamSynchronize(st));
        return RSV_OK;
    }
    if (on_device) {
        RSV_CUDA_TRY(launch_cast_f32_f64(st, v->n, (const float *)v->data, dst));
        return RSV_OK;
    }
    std::vector<float> tmp;
    try {
        tmp.resize(v->n);
    } catch (...) {
        return RSV_ENOMEM;
    }
    RSV_CUDA_TRY(cudaMemcpyAsync(tmp.data(), v->data, sizeof(float) * v->n, cudaMemcpyDeviceToHost, st));
    RSV_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < v->n; ++i) dst[i] = (double)tmp[i];
    return RSV_OK;
}

// ------------------------------------------------------------ vector algebra

static rsv_status reduce_once(void *stream, int64_t n, const double *x, const double *y, int sq, double *result) {
    if (n < 0 || (n > 0 && (!x || !y)) || !result) return RSV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    double *buf = nullptr;
    unsigned *cnt = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&buf, sizeof(double) * (kRedBlocks + 1) + 16, st);
    if (e != cudaSuccess) return cuda_status(e);
    cnt = (unsigned *)(buf + kRedBlocks + 1);
    double out = 0.0;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned), st)) == cudaSuccess &&
        (e = launch_dot<double>(st, n, x, y, buf, buf + kRedBlocks, cnt, sq, nullptr)) == cudaSuccess &&
        (e = cudaMemcpyAsync(&out, buf + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_status(e);
    *result = out;
    return RSV_OK;
}

rsv_status rsv_dot(void *stream, int64_t n, const double *x, const double *y, double *result) {
    return reduce_once(stream, n, x, y, 0, result);
}

rsv_status rsv_norm2(void *stream, int64_t n, const double *x, double *result) {
    return reduce_once(stream, n, x, x, 1, result);
}

rsv_status rsv_axpby(void *stream, int64_t n, double alpha, const double *x, double beta, const double *y,
                     double *z) {
    if (n < 0 || (n > 0 && (!x || !z || (beta != 0.0 && !y)))) return RSV_EINVAL;
    RSV_CUDA_TRY(launch_axpby<double>((cudaStream_t)stream, n, alpha, x, beta, y, z));
    return RSV_OK;
}

}  // extern "C"
