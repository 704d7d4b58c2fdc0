// C ABI of librsv: handles, argument checks and the Krylov drivers.
//
// Krylov solvers (Section "Solvers": restarted GMRES(m) and BiCGSTAB with
// the SOLVER fields rtol, atol, btol, maxit, restart).  All vector work and
// every solver scalar stay on the device; the host only launches kernels and
// reads a few status words once per GMRES cycle or every few BiCGSTAB
// iterations.  Kernels of a step that follows convergence see the device
// `done` flag and return at once.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace rsv {

static thread_local cudaError_t g_last_cuda = cudaSuccess;
static std::atomic<uint64_t> g_launches{0};
void set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

// ------------------------------------------------------------- tiny kernels

__global__ void gmres_cycle_init(DevState *ds) {
    ds->g[0] = ds->beta;
    for (int i = 1; i <= kMaxRestart; ++i) ds->g[i] = 0.0;
    ds->jend = 0;
    ds->done = 0;
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes, the
// previous Givens rotations, a new rotation and the residual estimate |g_{j+1}|.
__global__ void gmres_givens(DevState *ds, int j, int m) {
    if (ds->done) return;
    double *H = ds->H;
    for (int i = 0; i <= j; ++i) H[i * m + j] = ds->h1[i] + ds->h2[i];
    H[(j + 1) * m + j] = ds->hn;
    for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], b = H[(i + 1) * m + j];
        H[i * m + j] = ds->cs[i] * a + ds->sn[i] * b;
        H[(i + 1) * m + j] = -ds->sn[i] * a + ds->cs[i] * b;
    }
    const double a = H[j * m + j], b = H[(j + 1) * m + j];
    const double rho = hypot(a, b);
    if (!isfinite(rho) || !isfinite(ds->hn)) {
        if (ds->status == 0) ds->status = RSV_ENAN;
        ds->done = 1;
        return;
    }
    if (!(rho > 0.0)) {
        if (ds->status == 0) ds->status = RSV_EBREAKDOWN;
        ds->done = 1;
        return;
    }
    ds->cs[j] = a / rho;
    ds->sn[j] = b / rho;
    H[j * m + j] = rho;
    H[(j + 1) * m + j] = 0.0;
    ds->g[j + 1] = -ds->sn[j] * ds->g[j];
    ds->g[j] = ds->cs[j] * ds->g[j];
    ds->jend = j + 1;
    ds->iters += 1;
    const bool lucky = !(ds->hn > 0.0);
    if (fabs(ds->g[j + 1]) <= ds->tol || ds->iters >= ds->maxit || lucky || j + 1 == m) ds->done = 1;
}

__global__ void gmres_backsolve(DevState *ds, int m) {
    const int n = ds->jend;
    for (int i = n - 1; i >= 0; --i) {
        double s = ds->g[i];
        for (int q = i + 1; q < n; ++q) s -= ds->H[i * m + q] * ds->y[q];
        ds->y[i] = s / ds->H[i * m + i];
    }
}

// BiCGSTAB scalar steps (single thread).
__global__ void bicg_beta(DevState *ds, double btol) {
    if (ds->done) return;
    const double rho1 = ds->red[0];
    if (!isfinite(rho1)) { if (ds->status == 0) ds->status = RSV_ENAN; ds->done = 1; return; }
    if (fabs(rho1) <= btol * ds->red[8] * ds->red[9]) { if (ds->status == 0) ds->status = RSV_EBREAKDOWN; ds->done = 1; return; }
    ds->rho1 = rho1;
    ds->red[10] = (rho1 / ds->rho) * (ds->alpha / ds->omega);  // beta
}

__global__ void bicg_alpha(DevState *ds, double btol) {
    if (ds->done) return;
    const double rv = ds->red[1];
    if (!isfinite(rv)) { if (ds->status == 0) ds->status = RSV_ENAN; ds->done = 1; return; }
    if (fabs(rv) <= btol * ds->red[8] * ds->red[2]) { if (ds->status == 0) ds->status = RSV_EBREAKDOWN; ds->done = 1; return; }
    ds->alpha = ds->rho1 / rv;
}

__global__ void bicg_check_s(DevState *ds) {
    if (ds->done) return;
    ds->iters += 1;
    const double sn = ds->red[3];
    if (!isfinite(sn)) { if (ds->status == 0) ds->status = RSV_ENAN; ds->done = 1; return; }
    if (sn <= ds->tol) {
        ds->red[11] = 1.0;  // x += alpha ph pending
        ds->done = 1;
    }
}

__global__ void bicg_omega(DevState *ds, double btol) {
    if (ds->done) return;
    const double ts = ds->red[4], tt = ds->red[5];
    if (!(tt > 0.0) || !isfinite(tt)) { if (ds->status == 0) ds->status = isfinite(tt) ? RSV_EBREAKDOWN : RSV_ENAN; ds->done = 1; return; }
    const double om = ts / tt;
    if (fabs(om) <= btol) { if (ds->status == 0) ds->status = RSV_EBREAKDOWN; ds->done = 1; return; }
    ds->omega = om;
}

__global__ void bicg_finish_iter(DevState *ds) {
    if (ds->done) return;
    ds->rho = ds->rho1;
    const double rn = ds->red[9];
    if (!isfinite(rn)) { if (ds->status == 0) ds->status = RSV_ENAN; ds->done = 1; return; }
    if (rn <= ds->tol || ds->iters >= ds->maxit) ds->done = 1;
}

// p = r + beta (p - omega v)
__global__ void bicg_update_p(int64_t n, const DevState *ds, const double *r, const double *v, double *p) {
    if (ds->done) return;
    const double beta = ds->red[10], om = ds->omega;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        p[i] = r[i] + beta * (p[i] - om * v[i]);
}

// s = r - alpha v
__global__ void bicg_update_s(int64_t n, const DevState *ds, const double *r, const double *v, double *s) {
    if (ds->done) return;
    const double al = ds->alpha;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) s[i] = r[i] - al * v[i];
}

// x += alpha ph when the half step converged
__global__ void bicg_half_x(int64_t n, DevState *ds, const double *ph, double *x) {
    if (ds->red[11] != 1.0) return;
    const double al = ds->alpha;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) x[i] += al * ph[i];
}

__global__ void bicg_consume_half(DevState *ds) {
    if (ds->red[11] == 1.0) ds->red[11] = 2.0;
}

// x += alpha ph + omega sh; r = s - omega t
__global__ void bicg_update_xr(int64_t n, const DevState *ds, const double *ph, const double *sh,
                               const double *s, const double *t, double *x, double *r) {
    if (ds->done) return;
    const double al = ds->alpha, om = ds->omega;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        x[i] += al * ph[i] + om * sh[i];
        r[i] = s[i] - om * t[i];
    }
}

int egrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

rsv_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RSV_OK;
    set_last_cuda_error(e);
    return (e == cudaErrorMemoryAllocation) ? RSV_ENOMEM : RSV_ECUDA;
}

}  // namespace
}  // namespace rsv

using namespace rsv;

struct rsv_solver {
    rsv_mat *A = nullptr;
    rsv_solver_params p{};
    cudaStream_t st = nullptr;
    int64_t n = 0;
    int pc_type = -1;
    rsv_pc_params pcp{};
    uint64_t pc_version = ~0ull;
    DevState *ds = nullptr;
    double *partial = nullptr;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *t = nullptr;
    double *bv = nullptr;  // BiCGSTAB: r, rh, p, v, ph, sh, s, t (s and t adjacent)
    double *dinv = nullptr;
    double *d_b = nullptr, *d_x = nullptr;
    Schedule sch;
    IluTiles tiles;
    bool scratch_dirty = false;  // a sweep timed out: its sentinel scratch must be refilled
    double ms_setup = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

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
    if (A->d_rp) cudaFree(A->d_rp);
    if (A->d_ci) cudaFree(A->d_ci);
    if (A->d_v) cudaFree(A->d_v);
    if (A->d_v32) cudaFree(A->d_v32);
    delete A;
}

rsv_status rsv_mat_create(const rsv_grid *g, void *stream, rsv_mat **out) {
    if (!g || !out) return RSV_EINVAL;
    rsv_mat *A = new (std::nothrow) rsv_mat();
    if (!A) return RSV_ENOMEM;
    A->nx = g->nx;
    A->ny = g->ny;
    A->nz = g->nz;
    A->nb = (int64_t)g->nx * g->ny * g->nz;
    A->stream = (cudaStream_t)stream;
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    A->h_rp.resize(A->nb + 1);
    A->h_ci.reserve(7 * A->nb);
    A->h_rp[0] = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int32_t c = nx * ny * k + nx * j + i;
                if (k > 0) A->h_ci.push_back(c - nx * ny);
                if (j > 0) A->h_ci.push_back(c - nx);
                if (i > 0) A->h_ci.push_back(c - 1);
                A->h_ci.push_back(c);
                if (i < nx - 1) A->h_ci.push_back(c + 1);
                if (j < ny - 1) A->h_ci.push_back(c + nx);
                if (k < nz - 1) A->h_ci.push_back(c + nx * ny);
                A->h_rp[c + 1] = (int32_t)A->h_ci.size();
            }
    A->nnzb = (int64_t)A->h_ci.size();
    cudaError_t e;
    const size_t vbytes = sizeof(double) * (9 * (size_t)A->nnzb + 16);
    if ((e = cudaMalloc((void **)&A->d_rp, sizeof(int32_t) * (A->nb + 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&A->d_ci, sizeof(int32_t) * A->nnzb)) != cudaSuccess ||
        (e = cudaMalloc((void **)&A->d_v, vbytes)) != cudaSuccess ||
        (e = cudaMalloc((void **)&A->d_v32, vbytes / 2)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A->d_rp, A->h_rp.data(), sizeof(int32_t) * (A->nb + 1), cudaMemcpyHostToDevice,
                             A->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A->d_ci, A->h_ci.data(), sizeof(int32_t) * A->nnzb, cudaMemcpyHostToDevice,
                             A->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(A->d_v, 0, vbytes, A->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(A->d_v32, 0, vbytes / 2, A->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(A->stream)) != cudaSuccess) {
        mat_free(A);
        return cuda_status(e);
    }
    *out = A;
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
    RSV_CUDA_TRY(launch_cast_f64_f32(A->stream, 9 * A->nnzb, A->d_v, A->d_v32));
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
    if (!A || !x || !y) return RSV_EINVAL;
    RSV_CUDA_TRY(launch_spmv_f32(A, alpha, x, beta, y, nullptr));
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
        (e = launch_dot(st, n, x, y, buf, buf + kRedBlocks, cnt, sq, nullptr)) == cudaSuccess &&
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
    RSV_CUDA_TRY(launch_axpby((cudaStream_t)stream, n, alpha, x, beta, y, z));
    return RSV_OK;
}

// ------------------------------------------------------------------ solver

static void solver_free(rsv_solver *s) {
    if (!s) return;
    cudaStreamSynchronize(s->st);
    for (void *p : {(void *)s->ds, (void *)s->partial, (void *)s->V, (void *)s->Z, (void *)s->w, (void *)s->t,
                    (void *)s->bv, (void *)s->dinv, (void *)s->d_b, (void *)s->d_x})
        if (p) cudaFree(p);
    free_schedule(&s->sch);
    free_tiles(&s->tiles);
    if (s->e0) cudaEventDestroy(s->e0);
    if (s->e1) cudaEventDestroy(s->e1);
    delete s;
}

rsv_status rsv_solver_create(rsv_mat *A, const rsv_solver_params *p, rsv_solver **out) {
    if (!A || !p || !out) return RSV_EINVAL;
    if (p->solver < RSV_GMRES || p->solver > RSV_FGMRES) return RSV_EINVAL;
    if (p->restart < 1 || p->restart > kMaxRestart || p->maxit < 0 || !(p->rtol >= 0.0) || !(p->atol >= 0.0) ||
        !(p->btol >= 0.0) || p->watchdog < 1)
        return RSV_EINVAL;
    if (p->precision != RSV_PREC_FP64) return RSV_ENOTSUP;
    rsv_solver *s = new (std::nothrow) rsv_solver();
    if (!s) return RSV_ENOMEM;
    s->A = A;
    s->p = *p;
    s->st = A->stream;
    s->n = 3 * A->nb;
    const int64_t n = s->n;
    const int m = p->restart;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](double **ptr, size_t count) {
        if (e == cudaSuccess) e = cudaMalloc((void **)ptr, sizeof(double) * std::max<size_t>(count, 1));
    };
    e = cudaMalloc((void **)&s->ds, sizeof(DevState));
    alloc(&s->partial, (size_t)(kMaxRestart + 1) * kRedBlocks);
    if (p->solver == RSV_BICGSTAB) {
        alloc(&s->bv, 8 * (size_t)n);
    } else {
        alloc(&s->V, (size_t)(m + 1) * n);
        if (p->solver == RSV_FGMRES) alloc(&s->Z, (size_t)m * n);
    }
    alloc(&s->w, n);
    alloc(&s->t, n);
    alloc(&s->d_b, n);
    alloc(&s->d_x, n);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ds, 0, sizeof(DevState), s->st);
    if (e == cudaSuccess) e = cudaEventCreate(&s->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&s->e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
        solver_free(s);
        return cuda_status(e);
    }
    *out = s;
    return RSV_OK;
}

void rsv_solver_destroy(rsv_solver *s) { solver_free(s); }

static rsv_status read_status(rsv_solver *s, int *status) {
    RSV_CUDA_TRY(cudaMemcpyAsync(status, &s->ds->status, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

rsv_status rsv_precond_setup(rsv_solver *s, int pc_type, const rsv_pc_params *params) {
    if (!s || pc_type < RSV_PC_NONE || pc_type > RSV_PC_CPR) return RSV_EINVAL;
    rsv_pc_params pcp;
    rsv_pc_params_default(&pcp);
    if (params) pcp = *params;
    if (pc_type == RSV_PC_CPR) return RSV_ENOTSUP;
    rsv_mat *A = s->A;
    RSV_CUDA_TRY(cudaEventRecord(s->e0, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(&s->ds->status, 0, sizeof(int), s->st));
    if ((pc_type == RSV_PC_BJACOBI || pc_type == RSV_PC_BILU0) && !s->dinv)
        RSV_CUDA_TRY(cudaMalloc((void **)&s->dinv, sizeof(double) * 9 * std::max<int64_t>(A->nb, 1)));
    if (pc_type == RSV_PC_BJACOBI) RSV_CUDA_TRY(launch_bj_setup(A, s->dinv, &s->ds->status));
    if (pc_type == RSV_PC_BILU0) {
        if (!s->sch.cells) RSV_CUDA_TRY(build_schedule(A, &s->sch));
        RSV_CUDA_TRY(launch_ilu_setup(A, s->sch, s->dinv, &s->ds->status));
        RSV_CUDA_TRY(tiles_setup(A, s->dinv, &s->tiles));
    }
    RSV_CUDA_TRY(cudaEventRecord(s->e1, s->st));
    int status = 0;
    RSV_TRY(read_status(s, &status));
    float ms = 0.f;
    RSV_CUDA_TRY(cudaEventElapsedTime(&ms, s->e0, s->e1));
    s->ms_setup = ms;
    if (status != RSV_OK) {
        s->pc_type = -1;
        return (rsv_status)status;
    }
    s->pc_type = pc_type;
    s->pcp = pcp;
    s->pc_version = A->version;
    return RSV_OK;
}

// z = M^{-1} r on the solver stream; `done` gates the kernels.
static cudaError_t pc_apply(rsv_solver *s, const double *r, double *z, const int *done) {
    switch (s->pc_type) {
    case RSV_PC_NONE: return cudaMemcpyAsync(z, r, sizeof(double) * s->n, cudaMemcpyDeviceToDevice, s->st);
    case RSV_PC_BJACOBI: return launch_bj_apply(s->st, s->A->nb, s->dinv, r, z, done);
    case RSV_PC_BILU0:
        return launch_ilu_apply_tiles(s->A, s->tiles, r, z, done, &s->ds->status,
                                      (unsigned long long)s->p.watchdog * 1000ull);
    }
    return cudaErrorInvalidValue;
}

rsv_status rsv_precond_apply(rsv_solver *s, const double *r, double *z) {
    if (!s || !r || !z || r == z) return RSV_EINVAL;
    if (s->pc_type < 0 || s->pc_version != s->A->version) return RSV_EINVAL;
    RSV_CUDA_TRY(pc_apply(s, r, z, nullptr));
    return RSV_OK;
}

rsv_status rsv_precond_get_dinv(rsv_solver *s, double *dinv_host) {
    if (!s || !dinv_host || !s->dinv || (s->pc_type != RSV_PC_BJACOBI && s->pc_type != RSV_PC_BILU0))
        return RSV_EINVAL;
    RSV_CUDA_TRY(cudaMemcpyAsync(dinv_host, s->dinv, sizeof(double) * 9 * s->A->nb, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

// r = b - A x and ||r|| into *nrm (device)
static cudaError_t residual(rsv_solver *s, const double *b, const double *x, double *r, double *nrm) {
    cudaError_t e = cudaMemcpyAsync(r, b, sizeof(double) * s->n, cudaMemcpyDeviceToDevice, s->st);
    if (e == cudaSuccess) e = launch_spmv_f64(s->A, -1.0, x, 1.0, r, nullptr);
    if (e == cudaSuccess)
        e = launch_dot(s->st, s->n, r, r, s->partial, nrm, &s->ds->counter[0], 1, nullptr);
    return e;
}

struct HostState {
    double beta;
    int done, status, iters, jend;
};

static rsv_status fetch(rsv_solver *s, HostState *h) {
    DevState *ds = s->ds;
    RSV_CUDA_TRY(cudaMemcpyAsync(&h->beta, &ds->beta, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&h->done, &ds->done, 4 * sizeof(int), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

static rsv_status gmres_solve(rsv_solver *s, const double *b, double *x, double bnorm, rsv_solve_info *info) {
    const int64_t n = s->n;
    const int m = s->p.restart;
    const bool flex = s->p.solver == RSV_FGMRES;
    DevState *ds = s->ds;
    const double tol = std::max(s->p.rtol * bnorm, s->p.atol);
    int cycles = 0;
    HostState h{};
    rsv_status result = RSV_ENOCONV;
    for (;;) {
        RSV_CUDA_TRY(residual(s, b, x, s->V, &ds->beta));
        RSV_TRY(fetch(s, &h));
        if (h.status != RSV_OK) { result = (rsv_status)h.status; break; }
        if (!std::isfinite(h.beta)) { result = RSV_ENAN; break; }
        if (h.beta <= tol) { result = RSV_OK; break; }
        if (h.iters >= s->p.maxit) { result = RSV_ENOCONV; break; }
        ++cycles;
        rsv::count_launches(1);
        gmres_cycle_init<<<1, 1, 0, s->st>>>(ds);
        RSV_CUDA_TRY(launch_scale_inv(s->st, n, s->V, &ds->beta, nullptr));
        for (int j = 0; j < m; ++j) {
            double *vj = s->V + (size_t)j * n;
            double *w = s->V + (size_t)(j + 1) * n;
            double *z = flex ? s->Z + (size_t)j * n : s->t;
            RSV_CUDA_TRY(pc_apply(s, vj, z, &ds->done));
            RSV_CUDA_TRY(launch_spmv_f64(s->A, 1.0, z, 0.0, w, &ds->done));
            // classical Gram-Schmidt, two passes (re-orthogonalised)
            RSV_CUDA_TRY(launch_mdot(s->st, n, w, s->V, n, j + 1, s->partial, ds->h1, &ds->counter[0], &ds->done));
            RSV_CUDA_TRY(launch_maxpy(s->st, n, w, s->V, n, j + 1, ds->h1, -1.0, w, s->partial, nullptr,
                                      &ds->counter[1], &ds->done));
            RSV_CUDA_TRY(launch_mdot(s->st, n, w, s->V, n, j + 1, s->partial, ds->h2, &ds->counter[0], &ds->done));
            RSV_CUDA_TRY(launch_maxpy(s->st, n, w, s->V, n, j + 1, ds->h2, -1.0, w, s->partial, &ds->hn,
                                      &ds->counter[1], &ds->done));
            rsv::count_launches(1);
            gmres_givens<<<1, 1, 0, s->st>>>(ds, j, m);
            RSV_CUDA_TRY(launch_scale_inv(s->st, n, w, &ds->hn, &ds->done));
        }
        RSV_TRY(fetch(s, &h));
        if (h.status != RSV_OK && h.status != RSV_EBREAKDOWN) { result = (rsv_status)h.status; break; }
        if (h.jend > 0) {
            rsv::count_launches(1);
            gmres_backsolve<<<1, 1, 0, s->st>>>(ds, m);
            if (flex) {
                RSV_CUDA_TRY(launch_maxpy(s->st, n, x, s->Z, n, h.jend, ds->y, 1.0, x, s->partial, nullptr,
                                          &ds->counter[1], nullptr));
            } else {
                RSV_CUDA_TRY(launch_maxpy(s->st, n, nullptr, s->V, n, h.jend, ds->y, 1.0, s->w, s->partial, nullptr,
                                          &ds->counter[1], nullptr));
                RSV_CUDA_TRY(pc_apply(s, s->w, s->t, nullptr));
                RSV_CUDA_TRY(launch_axpby(s->st, n, 1.0, s->t, 1.0, x, x));
            }
        }
        if (h.status == RSV_EBREAKDOWN) { result = RSV_EBREAKDOWN; break; }
    }
    if (info) {
        info->iters = h.iters;
        info->restarts = cycles;
    }
    return result;
}

static rsv_status bicgstab_solve(rsv_solver *s, const double *b, double *x, double bnorm, rsv_solve_info *info) {
    const int64_t n = s->n;
    DevState *ds = s->ds;
    double *r = s->bv, *rh = r + n, *p = r + 2 * n, *v = r + 3 * n, *ph = r + 4 * n, *sh = r + 5 * n,
           *sv = r + 6 * n, *t = r + 7 * n;  // s (sv) and t adjacent: one two-column dot
    const double tol = std::max(s->p.rtol * bnorm, s->p.atol);
    const double btol = s->p.btol;
    RSV_CUDA_TRY(residual(s, b, x, r, &ds->red[9]));
    RSV_CUDA_TRY(cudaMemcpyAsync(rh, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&ds->red[8], &ds->red[9], sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(double) * n, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(double) * n, s->st));
    HostState h{};
    double rn0 = 0.0;
    RSV_CUDA_TRY(cudaMemcpyAsync(&rn0, &ds->red[9], sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    rsv_status result = RSV_ENOCONV;
    if (!std::isfinite(rn0)) return RSV_ENAN;
    if (rn0 <= tol) return RSV_OK;
    const double one = 1.0, zero = 0.0;
    RSV_CUDA_TRY(cudaMemcpyAsync(&ds->rho, &one, sizeof(double), cudaMemcpyHostToDevice, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&ds->alpha, &one, sizeof(double), cudaMemcpyHostToDevice, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&ds->omega, &one, sizeof(double), cudaMemcpyHostToDevice, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&ds->red[11], &zero, sizeof(double), cudaMemcpyHostToDevice, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    const int g = egrid(n);
    const int kBatch = 8;
    for (;;) {
        for (int it = 0; it < kBatch; ++it) {
            const int *done = &ds->done;
            RSV_CUDA_TRY(launch_dot(s->st, n, rh, r, s->partial, &ds->red[0], &ds->counter[0], 0, done));
            rsv::count_launches(1);
            bicg_beta<<<1, 1, 0, s->st>>>(ds, btol);
            rsv::count_launches(1);
            bicg_update_p<<<g, 256, 0, s->st>>>(n, ds, r, v, p);
            RSV_CUDA_TRY(pc_apply(s, p, ph, done));
            RSV_CUDA_TRY(launch_spmv_f64(s->A, 1.0, ph, 0.0, v, done));
            RSV_CUDA_TRY(launch_dot(s->st, n, rh, v, s->partial, &ds->red[1], &ds->counter[0], 0, done));
            RSV_CUDA_TRY(launch_dot(s->st, n, v, v, s->partial, &ds->red[2], &ds->counter[0], 1, done));
            rsv::count_launches(1);
            bicg_alpha<<<1, 1, 0, s->st>>>(ds, btol);
            rsv::count_launches(1);
            bicg_update_s<<<g, 256, 0, s->st>>>(n, ds, r, v, sv);
            RSV_CUDA_TRY(launch_dot(s->st, n, sv, sv, s->partial, &ds->red[3], &ds->counter[0], 1, done));
            rsv::count_launches(1);
            bicg_check_s<<<1, 1, 0, s->st>>>(ds);
            rsv::count_launches(1);
            bicg_half_x<<<g, 256, 0, s->st>>>(n, ds, ph, x);
            rsv::count_launches(1);
            bicg_consume_half<<<1, 1, 0, s->st>>>(ds);
            RSV_CUDA_TRY(pc_apply(s, sv, sh, done));
            RSV_CUDA_TRY(launch_spmv_f64(s->A, 1.0, sh, 0.0, t, done));
            RSV_CUDA_TRY(launch_mdot(s->st, n, t, sv, n, 2, s->partial, &ds->red[4], &ds->counter[0], done));
            rsv::count_launches(1);
            bicg_omega<<<1, 1, 0, s->st>>>(ds, btol);
            rsv::count_launches(1);
            bicg_update_xr<<<g, 256, 0, s->st>>>(n, ds, ph, sh, sv, t, x, r);
            RSV_CUDA_TRY(launch_dot(s->st, n, r, r, s->partial, &ds->red[9], &ds->counter[0], 1, done));
            rsv::count_launches(1);
            bicg_finish_iter<<<1, 1, 0, s->st>>>(ds);
        }
        RSV_CUDA_TRY(cudaGetLastError());
        RSV_TRY(fetch(s, &h));
        if (h.done || h.status != RSV_OK) {
            result = (h.status != RSV_OK) ? (rsv_status)h.status
                                          : (h.iters >= s->p.maxit ? RSV_ENOCONV : RSV_OK);
            break;
        }
    }
    if (result == RSV_ENOCONV && h.status == RSV_OK) {
        // stopped on maxit: report ENOCONV unless the last residual met the tolerance
        double rn = 0.0;
        RSV_CUDA_TRY(cudaMemcpyAsync(&rn, &ds->red[9], sizeof(double), cudaMemcpyDeviceToHost, s->st));
        RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
        if (rn <= tol) result = RSV_OK;
    }
    if (info) {
        info->iters = h.iters;
        info->restarts = 0;
    }
    return result;
}

rsv_status rsv_solve(rsv_solver *s, const double *b, double *x, int on_device, rsv_solve_info *info) {
    if (!s || !b || !x) return RSV_EINVAL;
    if (s->pc_type < 0 || s->pc_version != s->A->version) return RSV_EINVAL;
    const int64_t n = s->n;
    const double *db = b;
    double *dx = x;
    RSV_CUDA_TRY(cudaEventRecord(s->e0, s->st));
    if (!on_device) {
        RSV_CUDA_TRY(cudaMemcpyAsync(s->d_b, b, sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
        RSV_CUDA_TRY(cudaMemcpyAsync(s->d_x, x, sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
        db = s->d_b;
        dx = s->d_x;
    }
    // reset device state
    RSV_CUDA_TRY(cudaMemsetAsync(s->ds, 0, sizeof(DevState), s->st));
    if (s->scratch_dirty && s->tiles.scratch) {
        RSV_CUDA_TRY(reset_tiles_scratch(s->A, &s->tiles));
        s->scratch_dirty = false;
    }
    double bnorm = 0.0;
    RSV_CUDA_TRY(launch_dot(s->st, n, db, db, s->partial, &s->ds->bnorm, &s->ds->counter[0], 1, nullptr));
    RSV_CUDA_TRY(cudaMemcpyAsync(&bnorm, &s->ds->bnorm, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    if (!std::isfinite(bnorm)) return RSV_ENAN;
    const double tol = std::max(s->p.rtol * bnorm, s->p.atol);
    int maxit = s->p.maxit;
    RSV_CUDA_TRY(cudaMemcpyAsync(&s->ds->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&s->ds->maxit, &maxit, sizeof(int), cudaMemcpyHostToDevice, s->st));
    rsv_solve_info local{};
    rsv_status st = (s->p.solver == RSV_BICGSTAB) ? bicgstab_solve(s, db, dx, bnorm, &local)
                                                   : gmres_solve(s, db, dx, bnorm, &local);
    if (st == RSV_ECUDA || st == RSV_ENOMEM) return st;
    if (st == RSV_ETIMEOUT) s->scratch_dirty = true;
    // FP64 true residual, recomputed
    double rn = 0.0;
    RSV_CUDA_TRY(residual(s, db, dx, s->w, &s->ds->red[12]));
    RSV_CUDA_TRY(cudaMemcpyAsync(&rn, &s->ds->red[12], sizeof(double), cudaMemcpyDeviceToHost, s->st));
    if (!on_device) RSV_CUDA_TRY(cudaMemcpyAsync(x, s->d_x, sizeof(double) * n, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaEventRecord(s->e1, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    float ms = 0.f;
    RSV_CUDA_TRY(cudaEventElapsedTime(&ms, s->e0, s->e1));
    if (info) {
        info->iters = local.iters;
        info->restarts = local.restarts;
        info->outer_iters = 0;
        info->status = st;
        info->true_relres = bnorm > 0 ? rn / bnorm : rn;
        info->ms_setup = s->ms_setup;
        info->ms_solve = ms;
    }
    return st;
}

}  // extern "C"
