// Internal: the solver handle and helpers shared by the single-system
// drivers (solve.cu) and the batched driver (batch.cu).
#pragma once

#include "../../include/rsv_unet.h"
#include "common.cuh"

// Krylov workspace of one vector precision.
struct KrylovWork {
    void *V = nullptr;   // (m+1) basis vectors (GMRES) or 8 vectors (BiCGSTAB)
    void *Z = nullptr;   // m preconditioned vectors (FGMRES)
    void *w = nullptr;   // scratch
    void *t = nullptr;   // scratch
};

struct rsv_solver {
    rsv_mat *A = nullptr;
    rsv_solver_params p{};
    cudaStream_t st = nullptr;
    int64_t n = 0;
    int64_t ldv = 0;             // leading dimension of the Krylov vectors (n rounded up to 4)
    int pc_type = -1;
    rsv_pc_params pcp{};
    uint64_t pc_version = ~0ull;
    bool mixed = false;
    rsv::DevState *ds = nullptr;
    double *partial = nullptr;
    KrylovWork kw;               // FP64 work (FP64 solves) or FP32 work (mixed inner solves)
    double *r64 = nullptr;       // FP64 residual (true residual / refinement)
    double *d_b = nullptr, *d_x = nullptr;  // staging for host buffers
    float *rf = nullptr, *df = nullptr;     // mixed: scaled inner right-hand side and correction
    double *dinv = nullptr;      // FP64 inverted diagonal blocks (Jacobi: A_ii^-1, ILU: D_i^-1)
    float *dinv32 = nullptr;     // FP32 copy for mixed block Jacobi
    rsv::Schedule sch;
    rsv::IluTiles tiles;
    rsv::Cpr cpr;
    void *batch = nullptr;       // batched-solve state (batch.cu)
    // learned pressure stage (RSV_PC_CPR_LEARNED, learned.cu)
    rsv_unet *unet = nullptr;    // not owned
    double *lnk = nullptr;       // ln k of the cells, device
    int *lflags = nullptr;       // [0] fell back, [1] skip network, [2] skip V-cycle, [3] steps seen, [4] fallback iteration
    double *lhist = nullptr;     // the last implicit residual norms (ring of 64)
    int stall_window = 5;        // fall back when the residual fell by less than stall_drop
    double stall_drop = 0.10;    // over stall_window iterations
    // recorder of the pressure stage's right-hand sides (RSV_PC_CPR, FP64)
    double *rec_buf = nullptr;
    int rec_max = 0;
    int *rec_count = nullptr;
    double *acc = nullptr;       // accumulation blocks [nb][9] for true-IMPES decoupling, device
    double ms_setup = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace rsv {

// learned.cu: CPR with the network as pressure stage, CPR with recording, the stall watch.
cudaError_t learned_cpr_apply(rsv_solver *s, const double *f, double *x, const int *done);
cudaError_t cpr_apply_recording(rsv_solver *s, const double *f, double *x, const int *done);
cudaError_t learned_watch(rsv_solver *s, int j);
rsv_status learned_reset(rsv_solver *s);
rsv_status learned_finish(rsv_solver *s, int *fallback_iter);
void learned_free(rsv_solver *s);

template <typename T>
cudaError_t spmv(rsv_solver *s, T alpha, const T *x, T beta, T *y, const int *done);
template <>
inline cudaError_t spmv<double>(rsv_solver *s, double alpha, const double *x, double beta, double *y, const int *done) {
    return launch_spmv_f64(s->A, alpha, x, beta, y, done, &s->ds->status, (unsigned long long)s->p.watchdog * 1000ull);
}
template <>
inline cudaError_t spmv<float>(rsv_solver *s, float alpha, const float *x, float beta, float *y, const int *done) {
    return launch_spmv_f32(s->A, alpha, x, beta, y, done, &s->ds->status, (unsigned long long)s->p.watchdog * 1000ull);
}

// z = M^{-1} r on the solver stream in precision T; `done` gates the kernels.
template <typename T>
inline cudaError_t pc_apply(rsv_solver *s, const T *r, T *z, const int *done) {
    switch (s->pc_type) {
    case RSV_PC_NONE: return cudaMemcpyAsync(z, r, sizeof(T) * s->n, cudaMemcpyDeviceToDevice, s->st);
    case RSV_PC_BJACOBI:
        if (sizeof(T) == 8) return launch_bj_apply<T>(s->st, s->A->nb, (const T *)s->dinv, r, z, done);
        return launch_bj_apply<T>(s->st, s->A->nb, (const T *)s->dinv32, r, z, done);
    case RSV_PC_BILU0:
        return launch_ilu_apply_tiles<T>(s->A, s->tiles, r, z, done, &s->ds->status,
                                         (unsigned long long)s->p.watchdog * 1000ull);
    case RSV_PC_CPR:
        if (sizeof(T) == 8 && s->rec_buf)
            return cpr_apply_recording(s, (const double *)r, (double *)z, done);
        return cpr_apply<T>(s->A, s->cpr, s->tiles, r, z, done, &s->ds->status,
                            (unsigned long long)s->p.watchdog * 1000ull);
    case RSV_PC_CPR_LEARNED:
        if (sizeof(T) == 8) return learned_cpr_apply(s, (const double *)r, (double *)z, done);
        return cudaErrorInvalidValue;
    case RSV_PC_CPR_FP:
    case RSV_PC_CPR_FPF:
    case RSV_PC_CPR_FFPF:
        return cpr_apply_order<T>(s->A, s->cpr, s->tiles, cpr_stages(s->pc_type), r, z, done, &s->ds->status,
                                  (unsigned long long)s->p.watchdog * 1000ull);
    }
    return cudaErrorInvalidValue;
}

// r = b - A x and ||r|| into *nrm (device)
template <typename T>
inline cudaError_t residual(rsv_solver *s, const T *b, const T *x, T *r, double *nrm) {
    cudaError_t e = cudaMemcpyAsync(r, b, sizeof(T) * s->n, cudaMemcpyDeviceToDevice, s->st);
    if (e == cudaSuccess) e = spmv<T>(s, T(-1), x, T(1), r, nullptr);
    if (e == cudaSuccess) e = launch_dot<T>(s->st, s->n, r, r, s->partial, nrm, &s->ds->counter[0], 1, nullptr);
    return e;
}

void free_batch(rsv_solver *s);

}  // namespace rsv
