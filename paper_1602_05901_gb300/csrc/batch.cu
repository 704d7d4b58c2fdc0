// Batched solves: many independent reservoir systems of uneven grid sizes.
//
// The systems of a batch matrix (rsv_mat_create_batch) form one
// block-diagonal BSR matrix, so one SpMV launch and one cooperative launch of
// each block-ILU(0) tile sweep serve every system at once.  The Krylov
// method runs per system: right-preconditioned BiCGSTAB (Section "Solvers")
// with each system's own scalars (rho, alpha, omega, beta), its own
// convergence test and iteration count.  A converged system freezes: the
// vector updates skip its rows.  Segmented reductions give every system its
// own FP64-accurate dot products, deterministically (per system, partial
// sums of fixed chunks are added in chunk order by the last CTA to finish).
//
// One loop pass (two preconditioner applications, two SpMVs, four segmented
// reductions and the scalar steps) is captured once into a CUDA graph holding
// kGraphIters passes; the host replays the graph and reads a single
// "systems done" counter between replays.
//
// Mixed precision: an FP64 refinement loop per system (r = b - A x in FP64,
// per-system norms), FP32 inner BiCGSTAB on r / ||r|| to the inner
// tolerance, x += ||r|| d; systems that meet the outer tolerance stop.
//
// The SpMV tile shape (block rows per CTA) is picked by timing the candidates
// on the batch matrix at preconditioner setup.
#include <cmath>
#include <vector>

#include "reduce.cuh"
#include "solver.cuh"

namespace rsv {
namespace {

constexpr int kChunk = 8192;      // elements per reduction work item
constexpr int kGraphIters = 4;    // BiCGSTAB passes per graph replay
constexpr int kSegThreads = 256;
constexpr int kStallPasses = 30;  // FP32 inner solves: passes without progress before handing back

struct SegItem {
    int sys;
    int pad;
    int64_t begin, end;
};

// Per-system state of the batched BiCGSTAB (arrays of nsys).
struct BatchDev {
    double *rho, *rho1, *alpha, *omega, *beta, *tol, *rhn, *scale, *bnorm, *best;
    double *red;     // [8][nsys]: 0 <rh,r> 1 <rh,v> 2 ||v|| 3 ||s|| 4 <t,s> 5 <t,t> 6 ||r|| 7 spare
    int *done, *status, *iters, *half, *outer, *stall;
    int *ndone;      // systems done (single counter)
    unsigned *ticket;  // [4][nsys] reduction tickets
    double *partial;   // [2][nitems]
};

struct BatchState {
    int nsys = 0, nitems = 0;
    SegItem *items = nullptr;
    int *item_begin = nullptr;  // per system: first item; item_begin[nsys] = nitems
    BatchDev dv{};
    void *dev_block = nullptr;  // one allocation behind dv
    void *vec = nullptr;        // 8 Krylov vectors in the inner precision
    void *xin = nullptr;        // inner solution (FP64 mode: copy of x; mixed: the FP32 correction)
    void *rin = nullptr;        // inner right-hand side
    int *h_ndone = nullptr;     // pinned
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [0] FP64, [1] FP32
    size_t graph_nodes[2] = {0, 0};
    uint64_t graph_version = ~0ull;
    bool graph_ok[2] = {true, true};
    bool tuned = false;
    cudaStream_t own = nullptr;  // capture-capable stream used when the caller's is the legacy default
};

// Runs the batched solve on the solver's own stream when the caller's stream
// is the legacy default stream (which cannot be captured into a graph):
// the caller's stream is synchronised first and the handles point at the
// own stream until the solve returns.
struct StreamSwap {
    rsv_solver *s;
    cudaStream_t saved;
    bool active = false;
    StreamSwap(rsv_solver *s_, cudaStream_t own) : s(s_), saved(s_->st) {
        if (saved == nullptr || saved == cudaStreamLegacy) {
            cudaStreamSynchronize(saved);
            s->st = own;
            s->A->stream = own;
            active = true;
        }
    }
    ~StreamSwap() {
        if (active) {
            cudaStreamSynchronize(s->st);
            s->st = saved;
            s->A->stream = saved;
        }
    }
};

__device__ __forceinline__ int sys_of_elem(const int32_t *sys_of_cell, int64_t i) { return sys_of_cell[i / 3]; }

// out1[s] = <x, y1> (or its sqrt) and, when y2, out2[s] = <x, y2>, per system s.
template <typename T>
__global__ void __launch_bounds__(kSegThreads) seg_dot_kernel(const SegItem *__restrict__ items, int nitems,
                                                              const int *__restrict__ item_begin,
                                                              const T *__restrict__ x, const T *__restrict__ y1,
                                                              const T *__restrict__ y2, double *out1, double *out2,
                                                              int sqrt1, double *partial, unsigned *ticket,
                                                              const int *done) {
    __shared__ double sm[2][kSegThreads / 32];
    __shared__ bool last;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const SegItem w = items[it];
        Acc<T> a1, a2;
        if (!(done && done[w.sys])) {
            for (int64_t i = w.begin + threadIdx.x; i < w.end; i += blockDim.x) {
                const T xv = x[i];
                a1.add(xv, y1[i]);
                if (y2) a2.add(xv, y2[i]);
            }
        }
        double v1 = warp_sum(a1.value()), v2 = y2 ? warp_sum(a2.value()) : 0.0;
        if ((threadIdx.x & 31) == 0) {
            sm[0][threadIdx.x >> 5] = v1;
            sm[1][threadIdx.x >> 5] = v2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s1 = 0.0, s2 = 0.0;
            for (int q = 0; q < kSegThreads / 32; ++q) {
                s1 += sm[0][q];
                s2 += sm[1][q];
            }
            partial[it] = s1;
            partial[nitems + it] = s2;
            __threadfence();
            const unsigned nit = (unsigned)(item_begin[w.sys + 1] - item_begin[w.sys]);
            last = atomicAdd(&ticket[w.sys], 1u) == nit - 1;
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            double s1 = 0.0, s2 = 0.0;
            for (int q = item_begin[w.sys]; q < item_begin[w.sys + 1]; ++q) {
                s1 += __ldcg(&partial[q]);
                s2 += __ldcg(&partial[nitems + q]);
            }
            if (!(done && done[w.sys])) {
                out1[w.sys] = sqrt1 ? sqrt(s1) : s1;
                if (out2) out2[w.sys] = s2;
            }
            ticket[w.sys] = 0u;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void finish_sys(BatchDev d, int s, int code) {
    if (code && d.status[s] == 0) d.status[s] = code;
    if (!d.done[s]) {
        d.done[s] = 1;
        atomicAdd(d.ndone, 1);
    }
}

// BiCGSTAB scalar steps, one thread per system.
__global__ void b_beta(BatchDev d, int nsys, double btol) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || d.done[s]) return;
    const double rho1 = d.red[0 * nsys + s];
    if (!isfinite(rho1)) return finish_sys(d, s, RSV_ENAN);
    if (fabs(rho1) <= btol * d.rhn[s] * d.red[6 * nsys + s]) return finish_sys(d, s, RSV_EBREAKDOWN);
    d.rho1[s] = rho1;
    d.beta[s] = (rho1 / d.rho[s]) * (d.alpha[s] / d.omega[s]);
}

__global__ void b_alpha(BatchDev d, int nsys, double btol) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || d.done[s]) return;
    const double rv = d.red[1 * nsys + s], vn = sqrt(fmax(d.red[2 * nsys + s], 0.0));
    if (!isfinite(rv)) return finish_sys(d, s, RSV_ENAN);
    if (fabs(rv) <= btol * d.rhn[s] * vn) return finish_sys(d, s, RSV_EBREAKDOWN);
    d.alpha[s] = d.rho1[s] / rv;
}

__global__ void b_check_s(BatchDev d, int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || d.done[s]) return;
    d.iters[s] += 1;
    const double sn = d.red[3 * nsys + s];
    if (!isfinite(sn)) return finish_sys(d, s, RSV_ENAN);
    if (sn <= d.tol[s]) {
        d.half[s] = 1;  // x += alpha ph pending
        finish_sys(d, s, 0);
    }
}

__global__ void b_omega(BatchDev d, int nsys, double btol) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || d.done[s]) return;
    const double ts = d.red[4 * nsys + s], tt = d.red[5 * nsys + s];
    if (!isfinite(tt)) return finish_sys(d, s, RSV_ENAN);
    if (!(tt > 0.0)) return finish_sys(d, s, RSV_EBREAKDOWN);
    const double om = ts / tt;
    if (fabs(om) <= btol) return finish_sys(d, s, RSV_EBREAKDOWN);
    d.omega[s] = om;
}

// stall_limit > 0 (FP32 inner solves of refinement): a system whose residual
// has not dropped below 0.99 of its best for stall_limit passes ends its
// inner solve; FP32 BiCGSTAB can stagnate above the inner tolerance on an
// ill-conditioned system, and the FP64 outer step continues from there.
__global__ void b_finish(BatchDev d, int nsys, int maxit, int stall_limit) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || d.done[s]) return;
    d.rho[s] = d.rho1[s];
    const double rn = d.red[6 * nsys + s];
    if (!isfinite(rn)) return finish_sys(d, s, RSV_ENAN);
    if (rn <= d.tol[s]) return finish_sys(d, s, 0);
    if (d.iters[s] >= maxit) return finish_sys(d, s, RSV_ENOCONV);
    if (stall_limit > 0) {
        if (rn < 0.99 * d.best[s]) {
            d.best[s] = rn;
            d.stall[s] = 0;
        } else if (++d.stall[s] >= stall_limit) {
            return finish_sys(d, s, 0);
        }
    }
}

template <typename T>
__global__ void b_update_p(int64_t n, BatchDev d, const int32_t *__restrict__ soc, const T *r, const T *v, T *p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int s = sys_of_elem(soc, i);
        if (d.done[s]) continue;
        p[i] = r[i] + (T)d.beta[s] * (p[i] - (T)d.omega[s] * v[i]);
    }
}

template <typename T>
__global__ void b_update_s(int64_t n, BatchDev d, const int32_t *__restrict__ soc, const T *r, const T *v, T *sv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int s = sys_of_elem(soc, i);
        if (d.done[s]) continue;
        sv[i] = r[i] - (T)d.alpha[s] * v[i];
    }
}

template <typename T>
__global__ void b_half_x(int64_t n, BatchDev d, const int32_t *__restrict__ soc, const T *ph, T *x) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int s = sys_of_elem(soc, i);
        if (d.half[s] != 1) continue;
        x[i] += (T)d.alpha[s] * ph[i];
    }
}

__global__ void b_consume_half(BatchDev d, int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys && d.half[s] == 1) d.half[s] = 2;
}

template <typename T>
__global__ void b_update_xr(int64_t n, BatchDev d, const int32_t *__restrict__ soc, const T *ph, const T *sh,
                            const T *sv, const T *t, T *x, T *r) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int s = sys_of_elem(soc, i);
        if (d.done[s]) continue;
        const T al = (T)d.alpha[s], om = (T)d.omega[s];
        x[i] += al * ph[i] + om * sh[i];
        r[i] = sv[i] - om * t[i];
    }
}

// Start of an inner solve: per-system tolerance and scalars; systems marked
// finished by the outer loop stay frozen.
__global__ void b_init(BatchDev d, int nsys, double rtol_or_inner, int mixed, double rtol) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    d.rho[s] = d.alpha[s] = d.omega[s] = 1.0;
    d.half[s] = 0;
    d.rhn[s] = d.red[6 * nsys + s];
    // FP64 mode: tol = rtol ||b||.  Mixed: the inner right-hand side has unit norm; the
    // inner tolerance is inner_rtol, or less strict on the system's last outer step,
    // which only needs ||r|| below rtol ||b|| (factor 2 of margin).
    if (mixed) {
        const double rn = d.red[7 * nsys + s];
        double t = rtol_or_inner;
        if (rn > 0.0) t = fmax(t, 0.5 * rtol * d.bnorm[s] / rn);
        d.tol[s] = t;
    } else {
        d.tol[s] = rtol_or_inner * d.bnorm[s];
    }
    d.done[s] = d.outer[s];
    d.best[s] = d.red[6 * nsys + s];
    d.stall[s] = 0;
}

__global__ void b_count_done(BatchDev d, int nsys) {
    int c = 0;
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) c += d.done[s];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ int sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q];
        *d.ndone = t;
    }
}

// Outer-loop bookkeeping: systems whose FP64 residual meets rtol ||b|| are finished.
__global__ void b_outer_check(BatchDev d, int nsys, double rtol, const double *rn, int max_outer, int maxit) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || d.outer[s]) return;
    if (!isfinite(rn[s])) {
        d.outer[s] = 1;
        if (d.status[s] == 0) d.status[s] = RSV_ENAN;
    } else if (rn[s] <= rtol * d.bnorm[s]) {
        d.outer[s] = 1;
        d.status[s] = 0;
    } else if (d.scale[s] >= max_outer || d.iters[s] >= maxit) {
        d.outer[s] = 1;
        if (d.status[s] == 0 || d.status[s] == RSV_ENOCONV) d.status[s] = RSV_ENOCONV;
    } else {
        d.status[s] = 0;  // an inner breakdown or maxit leaves a usable correction
    }
}

template <typename T>
__global__ void b_scaled_copy(int64_t n, BatchDev d, const int32_t *__restrict__ soc, const double *__restrict__ r64,
                              const double *__restrict__ rn, T *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int s = sys_of_elem(soc, i);
        out[i] = d.outer[s] ? T(0) : (T)(r64[i] / rn[s]);
    }
}

__global__ void b_add_scaled(int64_t n, BatchDev d, const int32_t *__restrict__ soc, const float *__restrict__ df,
                             const double *__restrict__ rn, double *__restrict__ x) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int s = sys_of_elem(soc, i);
        if (!d.outer[s]) x[i] += rn[s] * (double)df[i];
    }
}

__global__ void b_bump_outer(BatchDev d, int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys && !d.outer[s]) d.scale[s] += 1.0;  // outer steps taken (kept as a double)
}

int egrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }
unsigned sgrid(int nsys) { return (unsigned)((nsys + 127) / 128); }

template <typename T>
cudaError_t seg_dot(rsv_solver *s, BatchState *B, const T *x, const T *y1, const T *y2, double *o1, double *o2,
                    int sqrt1, int slot, const int *done) {
    count_launches(1);
    const int grid = std::min(B->nitems, 4 * 152);
    seg_dot_kernel<T><<<grid, kSegThreads, 0, s->st>>>(B->items, B->nitems, B->item_begin, x, y1, y2, o1, o2, sqrt1,
                                                       B->dv.partial, B->dv.ticket + (size_t)slot * B->nsys, done);
    return cudaGetLastError();
}

template <typename T>
T *vecs(BatchState *B, int64_t ldv, int q) {
    return (T *)B->vec + (size_t)q * ldv;
}

// kGraphIters BiCGSTAB passes for all systems (the body that is captured).
template <typename T>
cudaError_t bicg_passes(rsv_solver *s, BatchState *B, T *x) {
    const int64_t n = s->n, ldv = s->ldv;
    const int nsys = B->nsys;
    const BatchDev d = B->dv;
    const int32_t *soc = s->A->d_sys_of_cell;
    T *r = vecs<T>(B, ldv, 0), *rh = vecs<T>(B, ldv, 1), *p = vecs<T>(B, ldv, 2), *v = vecs<T>(B, ldv, 3),
      *ph = vecs<T>(B, ldv, 4), *sh = vecs<T>(B, ldv, 5), *sv = vecs<T>(B, ldv, 6), *t = vecs<T>(B, ldv, 7);
    const double btol = s->p.btol;
    const int g = egrid(n);
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < kGraphIters && e == cudaSuccess; ++it) {
        count_launches(14);
        b_beta<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys, btol);
        b_update_p<T><<<g, 256, 0, s->st>>>(n, d, soc, r, v, p);
        if ((e = pc_apply<T>(s, p, ph, nullptr)) != cudaSuccess) break;
        if ((e = spmv<T>(s, T(1), ph, T(0), v, nullptr)) != cudaSuccess) break;
        if ((e = seg_dot<T>(s, B, v, rh, v, d.red + 1 * nsys, d.red + 2 * nsys, 0, 1, d.done)) != cudaSuccess) break;
        b_alpha<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys, btol);
        b_update_s<T><<<g, 256, 0, s->st>>>(n, d, soc, r, v, sv);
        if ((e = seg_dot<T>(s, B, sv, sv, (const T *)nullptr, d.red + 3 * nsys, nullptr, 1, 2, d.done)) !=
            cudaSuccess)
            break;
        b_check_s<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys);
        b_half_x<T><<<g, 256, 0, s->st>>>(n, d, soc, ph, x);
        b_consume_half<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys);
        if ((e = pc_apply<T>(s, sv, sh, nullptr)) != cudaSuccess) break;
        if ((e = spmv<T>(s, T(1), sh, T(0), t, nullptr)) != cudaSuccess) break;
        if ((e = seg_dot<T>(s, B, t, sv, t, d.red + 4 * nsys, d.red + 5 * nsys, 0, 3, d.done)) != cudaSuccess) break;
        b_omega<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys, btol);
        b_update_xr<T><<<g, 256, 0, s->st>>>(n, d, soc, ph, sh, sv, t, x, r);
        // ||r|| of the new residual and <rh, r> for the next pass, in one sweep
        if ((e = seg_dot<T>(s, B, r, r, rh, d.red + 6 * nsys, d.red + 0 * nsys, 1, 0, d.done)) != cudaSuccess) break;
        b_finish<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys, s->p.maxit, sizeof(T) == 4 ? kStallPasses : 0);
        b_count_done<<<1, 256, 0, s->st>>>(d, nsys);
        e = cudaGetLastError();
    }
    return e;
}

// Inner batched BiCGSTAB on A_T x = rhs (rhs, x in precision T), x from zero.
template <typename T>
rsv_status bicg_inner(rsv_solver *s, BatchState *B, const T *rhs, T *x, double tol_param, int mixed) {
    const int64_t n = s->n, ldv = s->ldv;
    const int nsys = B->nsys;
    const BatchDev d = B->dv;
    T *r = vecs<T>(B, ldv, 0), *rh = vecs<T>(B, ldv, 1), *p = vecs<T>(B, ldv, 2), *v = vecs<T>(B, ldv, 3);
    RSV_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(r, rhs, sizeof(T) * n, cudaMemcpyDeviceToDevice, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(rh, rhs, sizeof(T) * n, cudaMemcpyDeviceToDevice, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(T) * n, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(T) * n, s->st));
    // ||r|| and <rh, r> of the starting residual (no system is frozen yet for this sweep)
    RSV_CUDA_TRY(seg_dot<T>(s, B, r, r, rh, d.red + 6 * nsys, d.red + 0 * nsys, 1, 0, nullptr));
    count_launches(2);
    b_init<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys, tol_param, mixed, s->p.rtol);
    b_count_done<<<1, 256, 0, s->st>>>(d, nsys);
    RSV_CUDA_TRY(cudaGetLastError());
    const int gi = sizeof(T) == 8 ? 0 : 1;
    // (re)capture the graph of kGraphIters passes when the preconditioner changed
    if (B->graph_version != s->pc_version) {
        for (int q = 0; q < 2; ++q)
            if (B->graph[q]) {
                cudaGraphExecDestroy(B->graph[q]);
                B->graph[q] = nullptr;
            }
        B->graph_ok[0] = B->graph_ok[1] = true;
        B->graph_version = s->pc_version;
    }
    if (!B->graph[gi] && B->graph_ok[gi]) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t eb = bicg_passes<T>(s, B, x);
            e = cudaStreamEndCapture(s->st, &g);
            if (eb != cudaSuccess) e = eb;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph[gi], g, 0);
        if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &B->graph_nodes[gi]);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            // a stream that cannot be captured: launch the passes directly
            B->graph[gi] = nullptr;
            B->graph_ok[gi] = false;
            cudaGetLastError();
        }
    }
    const int max_rounds = s->p.maxit / kGraphIters + 2;
    for (int round = 0; round < max_rounds; ++round) {
        RSV_CUDA_TRY(cudaMemcpyAsync(B->h_ndone, d.ndone, sizeof(int), cudaMemcpyDeviceToHost, s->st));
        RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
        if (*B->h_ndone >= nsys) break;
        if (B->graph[gi]) {
            count_launches(B->graph_nodes[gi]);
            RSV_CUDA_TRY(cudaGraphLaunch(B->graph[gi], s->st));
        } else
            RSV_CUDA_TRY(bicg_passes<T>(s, B, x));
    }
    return RSV_OK;
}

// Segmented work items of the batch matrix (chunks of each system's unknowns).
rsv_status batch_init(rsv_solver *s, BatchState **out) {
    const rsv_mat *A = s->A;
    BatchState *B = new (std::nothrow) BatchState();
    if (!B) return RSV_ENOMEM;
    B->nsys = A->nsys;
    std::vector<SegItem> items;
    std::vector<int> ibeg;
    for (int q = 0; q < A->nsys; ++q) {
        ibeg.push_back((int)items.size());
        const int64_t b0 = 3 * A->h_sys[q].cell0;
        const int64_t b1 = (q + 1 < A->nsys) ? 3 * A->h_sys[q + 1].cell0 : 3 * A->nb;
        for (int64_t c = b0; c < b1; c += kChunk) items.push_back(SegItem{q, 0, c, std::min(c + kChunk, b1)});
    }
    ibeg.push_back((int)items.size());
    B->nitems = (int)items.size();
    const int ns = A->nsys;
    const size_t nd = 10 + 8;  // scalar double arrays + red[8]
    const size_t bytes = sizeof(double) * (nd * ns + 2 * (size_t)B->nitems) + sizeof(int) * (6 * ns + 4) +
                         sizeof(unsigned) * 4 * ns + 256;
    const size_t es = s->mixed ? sizeof(float) : sizeof(double);
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc((void **)&B->items, sizeof(SegItem) * items.size())) == cudaSuccess &&
        (e = cudaMalloc((void **)&B->item_begin, sizeof(int) * ibeg.size())) == cudaSuccess &&
        (e = cudaMalloc(&B->dev_block, bytes)) == cudaSuccess &&
        (e = cudaMalloc(&B->vec, 8 * (size_t)s->ldv * es)) == cudaSuccess &&
        (e = cudaMalloc(&B->xin, (size_t)s->ldv * es)) == cudaSuccess &&
        (e = cudaMalloc(&B->rin, (size_t)s->ldv * es)) == cudaSuccess &&
        (e = cudaMallocHost((void **)&B->h_ndone, sizeof(int))) == cudaSuccess &&
        (e = cudaMemcpyAsync(B->items, items.data(), sizeof(SegItem) * items.size(), cudaMemcpyHostToDevice,
                             s->st)) == cudaSuccess &&
        (e = cudaMemcpyAsync(B->item_begin, ibeg.data(), sizeof(int) * ibeg.size(), cudaMemcpyHostToDevice,
                             s->st)) == cudaSuccess &&
        (e = cudaMemsetAsync(B->dev_block, 0, bytes, s->st)) == cudaSuccess) {
        char *p = (char *)B->dev_block;
        auto take_d = [&](size_t cnt) { double *q = (double *)p; p += sizeof(double) * cnt; return q; };
        BatchDev &d = B->dv;
        d.rho = take_d(ns); d.rho1 = take_d(ns); d.alpha = take_d(ns); d.omega = take_d(ns); d.beta = take_d(ns);
        d.tol = take_d(ns); d.rhn = take_d(ns); d.scale = take_d(ns); d.bnorm = take_d(ns); d.best = take_d(ns);
        d.red = take_d(8 * (size_t)ns);
        d.partial = take_d(2 * (size_t)B->nitems);
        int *ip = (int *)p;
        d.done = ip; d.status = ip + ns; d.iters = ip + 2 * ns; d.half = ip + 3 * ns; d.outer = ip + 4 * ns;
        d.stall = ip + 5 * ns;
        d.ndone = ip + 6 * ns;
        d.ticket = (unsigned *)(ip + 6 * ns + 4);
        e = cudaStreamSynchronize(s->st);
    }
    if (e != cudaSuccess) {
        BatchState *tmp = B;
        s->batch = tmp;
        free_batch(s);
        return cuda_status(e);
    }
    *out = B;
    return RSV_OK;
}

}  // namespace

void free_batch(rsv_solver *s) {
    BatchState *B = (BatchState *)s->batch;
    if (!B) return;
    for (int q = 0; q < 2; ++q)
        if (B->graph[q]) cudaGraphExecDestroy(B->graph[q]);
    for (void *p : {(void *)B->items, (void *)B->item_begin, B->dev_block, B->vec, B->xin, B->rin})
        if (p) cudaFree(p);
    if (B->h_ndone) cudaFreeHost(B->h_ndone);
    if (B->own) cudaStreamDestroy(B->own);
    delete B;
    s->batch = nullptr;
}

}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_solve_batched(rsv_solver *s, const rsv_vec *b, rsv_vec *x, rsv_solve_info *infos) {
    if (!s || !b || !x) return RSV_EINVAL;
    if (b->prec != RSV_PREC_FP64 || x->prec != RSV_PREC_FP64 || b->n != s->n || x->n != s->n) return RSV_EINVAL;
    if (b->data == x->data && s->n > 0) return RSV_EINVAL;
    return rsv_solve_batched_ptr(s, (const double *)b->data, (double *)x->data, 1, infos);
}

extern "C" rsv_status rsv_solve_batched_ptr(rsv_solver *s, const double *b, double *x, int on_device,
                                            rsv_solve_info *infos) {
    if (!s || !b || !x) return RSV_EINVAL;
    if (s->pc_type < 0 || s->pc_version != s->A->version) return RSV_EINVAL;
    if (s->p.solver != RSV_BICGSTAB) return RSV_ENOTSUP;
    if (s->pc_type != RSV_PC_NONE && s->pc_type != RSV_PC_BJACOBI && s->pc_type != RSV_PC_BILU0) return RSV_ENOTSUP;
    rsv_mat *A = s->A;
    const int nsys = A->nsys;
    const int64_t n = s->n;
    if (!s->batch) RSV_TRY(batch_init(s, (BatchState **)&s->batch));
    BatchState *B = (BatchState *)s->batch;
    if (!B->own) RSV_CUDA_TRY(cudaStreamCreateWithFlags(&B->own, cudaStreamNonBlocking));
    StreamSwap swap(s, B->own);
    if (!B->tuned) {
        RSV_CUDA_TRY(spmv_autotune(A));
        B->tuned = true;
    }
    const BatchDev d = B->dv;
    RSV_CUDA_TRY(cudaEventRecord(s->e0, s->st));
    const double *db = b;
    double *dx = x;
    if (!on_device) {
        RSV_CUDA_TRY(cudaMemcpyAsync(s->d_b, b, sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
        RSV_CUDA_TRY(cudaMemcpyAsync(s->d_x, x, sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
        db = s->d_b;
        dx = s->d_x;
    }
    // per-system state from scratch; ||b|| per system
    RSV_CUDA_TRY(cudaMemsetAsync(d.done, 0, sizeof(int) * (6 * nsys + 4), s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(d.scale, 0, sizeof(double) * nsys, s->st));
    RSV_CUDA_TRY(seg_dot<double>(s, B, db, db, (const double *)nullptr, d.bnorm, nullptr, 1, 0, nullptr));
    if (!s->mixed) {
        // FP64: BiCGSTAB on A x = b from the given x (solve for the correction of b - A x0)
        double *r0 = s->r64;
        RSV_CUDA_TRY(cudaMemcpyAsync(r0, db, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->st));
        RSV_CUDA_TRY(launch_spmv_f64(A, -1.0, dx, 1.0, r0, nullptr, &s->ds->status, (unsigned long long)s->p.watchdog * 1000ull));
        RSV_TRY(bicg_inner<double>(s, B, r0, (double *)B->xin, s->p.rtol, 0));
        RSV_CUDA_TRY(launch_axpby<double>(s->st, n, 1.0, (const double *)B->xin, 1.0, dx, dx));
    } else {
        double *rn = d.red + 7 * nsys;  // outer residual norms
        for (int outer = 0; outer <= s->p.max_outer; ++outer) {
            RSV_CUDA_TRY(cudaMemcpyAsync(s->r64, db, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->st));
            RSV_CUDA_TRY(launch_spmv_f64(A, -1.0, dx, 1.0, s->r64, nullptr, &s->ds->status, (unsigned long long)s->p.watchdog * 1000ull));
            RSV_CUDA_TRY(seg_dot<double>(s, B, s->r64, s->r64, (const double *)nullptr, rn, nullptr, 1, 0, nullptr));
            count_launches(1);
            b_outer_check<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys, s->p.rtol, rn, s->p.max_outer, s->p.maxit);
            // all finished?
            count_launches(1);
            BatchDev od = d;
            od.done = d.outer;  // count the systems the outer loop has finished
            b_count_done<<<1, 256, 0, s->st>>>(od, nsys);
            RSV_CUDA_TRY(cudaMemcpyAsync(B->h_ndone, d.ndone, sizeof(int), cudaMemcpyDeviceToHost, s->st));
            RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
            if (*B->h_ndone >= nsys) break;
            count_launches(2);
            b_scaled_copy<float><<<egrid(n), 256, 0, s->st>>>(n, d, A->d_sys_of_cell, s->r64, rn, (float *)B->rin);
            b_bump_outer<<<sgrid(nsys), 128, 0, s->st>>>(d, nsys);
            RSV_TRY(bicg_inner<float>(s, B, (const float *)B->rin, (float *)B->xin, s->p.inner_rtol, 1));
            count_launches(1);
            b_add_scaled<<<egrid(n), 256, 0, s->st>>>(n, d, A->d_sys_of_cell, (const float *)B->xin, rn, dx);
            RSV_CUDA_TRY(cudaGetLastError());
        }
    }
    // FP64 true residual per system
    double *rn = d.red + 7 * nsys;
    RSV_CUDA_TRY(cudaMemcpyAsync(s->r64, db, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->st));
    RSV_CUDA_TRY(launch_spmv_f64(A, -1.0, dx, 1.0, s->r64, nullptr, &s->ds->status, (unsigned long long)s->p.watchdog * 1000ull));
    RSV_CUDA_TRY(seg_dot<double>(s, B, s->r64, s->r64, (const double *)nullptr, rn, nullptr, 1, 0, nullptr));
    std::vector<double> h_rn(nsys), h_bn(nsys), h_outer(nsys);
    std::vector<int> h_iters(nsys), h_status(nsys);
    RSV_CUDA_TRY(cudaMemcpyAsync(h_rn.data(), rn, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(h_bn.data(), d.bnorm, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(h_outer.data(), d.scale, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(h_iters.data(), d.iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(h_status.data(), d.status, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s->st));
    if (!on_device) RSV_CUDA_TRY(cudaMemcpyAsync(x, s->d_x, sizeof(double) * n, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaEventRecord(s->e1, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    float ms = 0.f;
    RSV_CUDA_TRY(cudaEventElapsedTime(&ms, s->e0, s->e1));
    rsv_status worst = RSV_OK;
    for (int q = 0; q < nsys; ++q) {
        const double rel = h_bn[q] > 0 ? h_rn[q] / h_bn[q] : h_rn[q];
        int st = h_status[q];
        if (st == RSV_OK && !(rel <= s->p.rtol || h_rn[q] <= s->p.atol)) st = RSV_ENOCONV;
        if (st == RSV_EBREAKDOWN && (rel <= s->p.rtol)) st = RSV_OK;
        if (infos) {
            infos[q].iters = h_iters[q];
            infos[q].restarts = 0;
            infos[q].outer_iters = (int)h_outer[q];
            infos[q].status = st;
            infos[q].true_relres = rel;
            infos[q].ms_setup = s->ms_setup;
            infos[q].ms_solve = ms;
            infos[q].fallback_iter = -1;
        }
        if (st != RSV_OK && worst == RSV_OK) worst = (rsv_status)st;
    }
    return worst;
}
