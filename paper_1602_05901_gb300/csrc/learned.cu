// CPR with a learned pressure stage, and the recorder of the pressure stage's
// inputs that provides its training samples.
//
// The paper's CPR preconditioner (Section "CPR", two-stage form) first solves
// the decoupled pressure system for the restricted residual, then corrects
// the full system with block ILU(0).  Here the first stage runs the U-Net
// (unet.cu) on the restricted residual instead of the multigrid V-cycle.
// Both pressure solvers are launched on every application; device flags let
// exactly one of them run, so falling back to the V-cycle needs no host round
// trip:
//   skip_net = done || fell_back,  skip_vcycle = done || !fell_back.
// The solve falls back (for good) when the network's output holds a NaN or an
// Inf, or when the implicit residual norm of FGMRES falls by less than a
// fraction `drop` over `window` consecutive iterations (default 10% over 5).
#include <cmath>

#include "solver.cuh"
#include "unet.cuh"

namespace rsv {
namespace {

int blocks_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1 << 20)); }

__global__ void gates_kernel(const int *done, int *fl) {
    const int d = done ? *done : 0;
    fl[1] = (d || fl[0]) ? 1 : 0;
    fl[2] = (d || !fl[0]) ? 1 : 0;
}

// Any NaN or Inf in the network's correction: fall back, in this very application.
__global__ void check_finite(const double *__restrict__ x, int64_t n, int *fl, const int *iters) {
    if (fl[1]) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || isfinite(x[i])) return;
    if (atomicCAS(&fl[0], 0, 1) == 0) fl[4] = *iters;
}

constexpr int kHist = 64;  // ring of implicit residual norms; the stall window is at most kHist

// After the Givens rotation of Arnoldi step j: the implicit residual |g[j+1]|.
// Stall: it fell by less than the fraction `drop` over the last `window` steps.
__global__ void watch_kernel(const DevState *ds, int j, int *fl, double *hist, int window, double drop) {
    if (ds->jend != j + 1 || fl[0]) return;  // the step did not run, or the solve already fell back
    const double r = fabs(ds->g[j + 1]);
    const int k = fl[3];
    if (!isfinite(r) || (k >= window && r > (1.0 - drop) * hist[(k - window) % kHist])) {
        fl[0] = 1;
        fl[4] = ds->iters;
    }
    hist[k % kHist] = r;
    fl[3] = k + 1;
}

__global__ void reset_kernel(int *fl) {
    fl[0] = fl[1] = fl[2] = fl[3] = 0;
    fl[4] = -1;
}

// Recorder: copy p into slot *count (if not done and below max), then bump the count.
__global__ void record_copy(const double *__restrict__ p, int64_t nb, double *__restrict__ buf, int max,
                            const int *count, const int *done) {
    if (done && *done) return;
    const int k = *count;
    if (k >= max) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nb) buf[(int64_t)k * nb + i] = p[i];
}
__global__ void record_bump(int *count, int max, const int *done) {
    if ((done && *done) || *count >= max) return;
    *count += 1;
}

}  // namespace

cudaError_t learned_cpr_apply(rsv_solver *s, const double *f, double *x, const int *done) {
    const rsv_mat *A = s->A;
    cudaStream_t st = A->stream;
    const Cpr &P = s->cpr;
    int *fl = s->lflags;
    cudaError_t e = cpr_restrict<double>(A, P, f, done);
    if (e != cudaSuccess) return e;
    gates_kernel<<<1, 1, 0, st>>>(done, fl);
    if (unet_apply_device(s->unet, st, (const double *)P.b[0], s->lnk, (double *)P.x[0], &fl[1]) != RSV_OK)
        return cudaErrorLaunchFailure;
    check_finite<<<blocks_of(A->nb), 256, 0, st>>>((const double *)P.x[0], A->nb, fl, &s->ds->iters);
    gates_kernel<<<1, 1, 0, st>>>(done, fl);
    count_launches(3);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cpr_pressure_vcycle<double>(A, P, &fl[2]);
    if (e == cudaSuccess)
        e = cpr_finish<double>(A, P, s->tiles, f, x, done, &s->ds->status, (unsigned long long)s->p.watchdog * 1000ull);
    return e;
}

cudaError_t cpr_apply_recording(rsv_solver *s, const double *f, double *x, const int *done) {
    const rsv_mat *A = s->A;
    cudaStream_t st = A->stream;
    const Cpr &P = s->cpr;
    cudaError_t e = cpr_restrict<double>(A, P, f, done);
    if (e != cudaSuccess) return e;
    record_copy<<<blocks_of(A->nb), 256, 0, st>>>((const double *)P.b[0], A->nb, s->rec_buf, s->rec_max, s->rec_count,
                                                  done);
    record_bump<<<1, 1, 0, st>>>(s->rec_count, s->rec_max, done);
    count_launches(2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cpr_pressure_vcycle<double>(A, P, done);
    if (e == cudaSuccess)
        e = cpr_finish<double>(A, P, s->tiles, f, x, done, &s->ds->status, (unsigned long long)s->p.watchdog * 1000ull);
    return e;
}

cudaError_t learned_watch(rsv_solver *s, int j) {
    watch_kernel<<<1, 1, 0, s->st>>>(s->ds, j, s->lflags, s->lhist, s->stall_window, s->stall_drop);
    count_launches(1);
    return cudaGetLastError();
}

rsv_status learned_reset(rsv_solver *s) {
    reset_kernel<<<1, 1, 0, s->st>>>(s->lflags);
    count_launches(1);
    RSV_CUDA_TRY(cudaGetLastError());
    return RSV_OK;
}

// The fallback iteration of the solve just finished, and the network's device error word.
rsv_status learned_finish(rsv_solver *s, int *fallback_iter) {
    RSV_CUDA_TRY(cudaMemcpyAsync(fallback_iter, &s->lflags[4], sizeof(int), cudaMemcpyDeviceToHost, s->st));
    const int err = unet_error(s->unet, s->st);  // synchronises
    return err ? (rsv_status)err : RSV_OK;
}

void learned_free(rsv_solver *s) {
    for (void *p : {(void *)s->lnk, (void *)s->lflags, (void *)s->lhist, (void *)s->rec_count})
        if (p) cudaFree(p);
    s->lnk = nullptr;
    s->lflags = nullptr;
    s->lhist = nullptr;
    s->rec_count = nullptr;
}

}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_solver_set_learned(rsv_solver *s, rsv_unet *u, const double *lnk, int on_device,
                                             int stall_window, double stall_drop) {
    if (!s || !u || !lnk || stall_window > kHist || !(stall_drop < 1.0)) return RSV_EINVAL;
    const rsv_mat *A = s->A;
    int nx, ny, nz;
    unet_dims(u, &nx, &ny, &nz);
    if (A->nsys != 1 || A->h_sys[0].nx != nx || A->h_sys[0].ny != ny || A->h_sys[0].nz != nz) return RSV_EINVAL;
    if (!s->lnk) RSV_CUDA_TRY(cudaMalloc((void **)&s->lnk, sizeof(double) * A->nb));
    if (!s->lflags) RSV_CUDA_TRY(cudaMalloc((void **)&s->lflags, sizeof(int) * 8));
    if (!s->lhist) RSV_CUDA_TRY(cudaMalloc((void **)&s->lhist, sizeof(double) * kHist));
    RSV_CUDA_TRY(cudaMemcpyAsync(s->lnk, lnk, sizeof(double) * A->nb,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
    RSV_TRY(learned_reset(s));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    s->unet = u;
    s->stall_window = stall_window > 0 ? stall_window : 5;
    s->stall_drop = stall_window > 0 ? stall_drop : 0.10;
    return RSV_OK;
}

extern "C" rsv_status rsv_solver_record_pressure(rsv_solver *s, double *buf, int max_samples) {
    if (!s || (buf && max_samples < 1)) return RSV_EINVAL;
    if (!s->rec_count) RSV_CUDA_TRY(cudaMalloc((void **)&s->rec_count, sizeof(int)));
    RSV_CUDA_TRY(cudaMemsetAsync(s->rec_count, 0, sizeof(int), s->st));
    s->rec_buf = buf;
    s->rec_max = buf ? max_samples : 0;
    return RSV_OK;
}

extern "C" rsv_status rsv_solver_recorded(rsv_solver *s, int *count) {
    if (!s || !count) return RSV_EINVAL;
    *count = 0;
    if (!s->rec_count) return RSV_OK;
    RSV_CUDA_TRY(cudaMemcpyAsync(count, s->rec_count, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}
