// C ABI of librsv, part 2: the solver handle, preconditioner setup/apply and
// the Krylov drivers.
//
// Krylov solvers (Section "Solvers": restarted GMRES(m) and BiCGSTAB with the
// SOLVER fields rtol, atol, btol, maxit, restart).  All vector work and every
// solver scalar stay on the device; the host only launches kernels and reads
// a few status words once per GMRES cycle or every few BiCGSTAB iterations.
// Kernels of a step that follows convergence see the device `done` flag and
// return at once.
//
// Arnoldi orthogonalisation is classical Gram-Schmidt with one reorthogonalisation
// ("all projections, then one multi-vector update", twice).  FP64 bases take the
// second pass's projections from the Gram matrix of the basis (see
// gmres_gram_step), so a step reads the basis twice.  FP32 bases (GMRES) delay
// the second pass by one step and take it in the same read of the basis as the
// next step's projections (gmres_dcgs2_step), which keeps the second pass acting
// on the stored FP32 vector: two reads of the basis per step.  FP32 FGMRES runs
// the second pass explicitly when the first one cancelled more than 1 - 1/sqrt(2)
// of the norm.  The Hessenberg columns, Givens rotations and the residual estimate
// are FP64 scalars kept in device memory.
//
// Mixed precision (precision = RSV_PREC_MIXED): an FP64 iterative-refinement
// loop r = b - A x (FP64 SpMV, FP64 norm), inner solve A d = r / ||r|| with
// FP32 matrix values, FP32 preconditioner factors and an FP32 Krylov basis
// (dot products still accumulate in FP64), then x += ||r|| d.
#include <cmath>
#include <new>
#include <vector>

#include "solver.cuh"

namespace rsv {
namespace {

// ------------------------------------------------------------- tiny kernels

__global__ void gmres_cycle_init(DevState *ds) {
    ds->g[0] = ds->beta;
    for (int i = 1; i <= kMaxRestart; ++i) ds->g[i] = 0.0;
    ds->jend = 0;
    ds->conv = 0;
    ds->done = 0;
}

__device__ __forceinline__ void raise_status(DevState *ds, int code) {
    if (ds->status == 0) ds->status = code;
    ds->done = 1;
}

// Givens step on column j of the Hessenberg matrix, staged in shared memory as col[0..j+1]
// with the previous rotations in cs/sn: the previous rotations, a new rotation, the
// residual estimate |g_{j+1}| and the stopping test.  Thread 0 runs the serial chain at
// shared-memory latency; then the block stores the rotated column.  Called by the whole block.
__device__ void rotate_column(DevState *ds, double *col, const double *cs, const double *sn, int j, int m) {
    double *H = ds->H;
    const int t = threadIdx.x;
    if (t == 0) {
        for (int i = 0; i < j; ++i) {
            const double a = col[i], b = col[i + 1];
            col[i] = cs[i] * a + sn[i] * b;
            col[i + 1] = -sn[i] * a + cs[i] * b;
        }
        const double a = col[j], b = col[j + 1];
        const double rho = hypot(a, b);
        // b = col[j+1], the subdiagonal entry (a norm, >= 0): no earlier rotation touches it
        if (!isfinite(rho) || !isfinite(b)) {
            raise_status(ds, RSV_ENAN);
        } else if (!(rho > 0.0)) {
            raise_status(ds, RSV_EBREAKDOWN);
        } else {
            ds->cs[j] = a / rho;
            ds->sn[j] = b / rho;
            H[j * m + j] = rho;
            H[(j + 1) * m + j] = 0.0;
            ds->g[j + 1] = -ds->sn[j] * ds->g[j];
            ds->g[j] = ds->cs[j] * ds->g[j];
            ds->jend = j + 1;
            ds->iters += 1;
            const bool lucky = !(b > 0.0);
            const bool met = fabs(ds->g[j + 1]) <= ds->tol;
            if (met || lucky) ds->conv = 1;
            if (met || ds->iters >= ds->maxit || lucky || j + 1 == m) ds->done = 1;
        }
    }
    __syncthreads();
    for (int i = t; i < j; i += blockDim.x) H[i * m + j] = col[i];
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes (h1 + h2, and
// ||w|| after them as the subdiagonal entry), then its Givens step.
__global__ void gmres_givens(DevState *ds, int j, int m) {
    if (ds->done) return;
    __shared__ double col[kMaxRestart + 1], cs[kMaxRestart], sn[kMaxRestart];
    const int t = threadIdx.x;
    for (int i = t; i <= j; i += blockDim.x) col[i] = ds->h1[i] + ds->h2[i];
    for (int i = t; i < j; i += blockDim.x) {
        cs[i] = ds->cs[i];
        sn[i] = ds->sn[i];
    }
    if (t == 0) col[j + 1] = ds->hn;
    __syncthreads();
    rotate_column(ds, col, cs, sn, j, m);
}

// One step of GMRES's Arnoldi process by classical Gram-Schmidt with delayed
// reorthogonalisation (the FP32 basis of the inner solves).  Step j holds the final
// v_0..v_{j-1}, u_j (the once-orthogonalised, unnormalised vector of step j-1; u_0 = r)
// and w = A M^{-1} u_j, and the multi-dot gave ou = V_{0..j}^T u_j and ow = V_{0..j}^T w
// (V_j = u_j).  With s = ou[0..j-1] and rho^2 = <u_j,u_j> - s.s:
//   v_j = (u_j - V s) / rho, so Hessenberg column j-1 becomes [h1 + s; rho]: its
//   Givens step and stopping test run here (one step late; a step that finds its
//   predecessor converged leaves its own product unused);
//   A M^{-1} V_{0..j-1} = V_{0..j} Hbar (the Arnoldi relation) gives
//   A M^{-1} v_j = (w - V_{0..j} Hbar s) / rho, whose projections on V_{0..j} are
//   y = ([t; (c - s.t)/rho] - Hbar s) / rho (t = ow[0..j-1], c = ow[j]).  y is
//   column j's first pass (h1), and the update pass forms v_j and
//   u_{j+1} = A M^{-1} v_j - V_{0..j} y from the stored u_j and w with the
//   coefficients cB, cS[0] (v_j) and cA, cS[1], cS[0] (u_{j+1}).
// final: the cycle's last step finalises column j-1 only (no w).  Each step reads the
// basis twice (multi-dot and update), against three times for two explicit passes.
// One block of 128 threads.
__global__ void gmres_dcgs2_step(DevState *ds, int j, int m, int final_only) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (ds->done) return;
    constexpr int L = kMaxRestart + 1;
    __shared__ double s[L], tv[L], col[L], cs[kMaxRestart], sn[kMaxRestart], hs[L], red[2];
    __shared__ int stop;
    const int t = threadIdx.x;
    if (t < j) {
        s[t] = ds->ou[t];
        tv[t] = final_only ? 0.0 : ds->ow[t];
    }
    __syncthreads();
    if (t == 0) {
        double ss = 0.0, st = 0.0;
        for (int q = 0; q < j; ++q) {
            ss += s[q] * s[q];
            st += s[q] * tv[q];
        }
        red[0] = ss;
        red[1] = st;
    }
    __syncthreads();
    const double rho2 = ds->ou[j] - red[0];
    const double rho = rho2 > 0.0 ? sqrt(rho2) : (rho2 == rho2 ? 0.0 : rho2);  // NaN stays NaN
    if (j == 0) {
        if (t == 0) {
            ds->g[0] = rho;  // u_0 = r: rho = ||r||
            if (!isfinite(rho)) raise_status(ds, RSV_ENAN);
            else if (!(rho > 0.0)) raise_status(ds, RSV_EBREAKDOWN);
        }
    } else {
        if (t < j) col[t] = ds->h1[t] + s[t];
        if (t < j - 1) {
            cs[t] = ds->cs[t];
            sn[t] = ds->sn[t];
        }
        if (t == 0) col[j] = rho;
        __syncthreads();
        if (t <= j) ds->Hu[t * m + (j - 1)] = col[t];
        __syncthreads();
        rotate_column(ds, col, cs, sn, j - 1, m);
    }
    __syncthreads();
    if (t == 0) stop = ds->done;
    __syncthreads();
    if (final_only || stop) return;
    const double ri = 1.0 / rho;
    if (t <= j) {  // (Hbar s)_t over the finalised columns 0..j-1 (Hbar is upper Hessenberg)
        double h = 0.0;
        for (int c = t > 0 ? t - 1 : 0; c < j; ++c) h += ds->Hu[t * m + c] * s[c];
        hs[t] = h;
    }
    __syncthreads();
    const double yj = (ds->ow[j] - red[1]) * ri * ri - hs[j] * ri;
    const double e = hs[j] * ri + yj;
    if (t < j) {
        const double yq = (tv[t] - hs[t]) * ri;
        ds->h1[t] = yq;
        ds->cA[t] = ri * hs[t] + yq - e * ri * s[t];
        ds->cB[t] = s[t] * ri;
    }
    if (t == 0) {
        ds->h1[j] = yj;
        ds->cS[0] = ri;
        ds->cS[1] = e * ri;
    }
}

// Classical Gram-Schmidt with its second pass taken from the Gram matrix G = V^T V
// of the basis.  With h1 = V^T w, the second pass's projections of w' = w - V h1
// are V^T w' = h1 - G h1, so the two passes together subtract V h with
// h = h1 + (h1 - G h1); G's new column <v_j, V> comes from the same read of the
// basis as h1.  Column j of G (i <= j) is stored, G kept symmetric, h written to
// h1 and h2 cleared (the Hessenberg column is h1 + h2).  One block of kMaxRestart
// + 1 threads.  Used for FP64 bases.
// After the first Gram-Schmidt pass of an FP32 basis: keep its result when
// ||w'|| >= ||w|| / sqrt(2), otherwise run the second pass (its coefficients add
// to the first pass's).
__global__ void gmres_reorth_check(DevState *ds, int k) {
    if (ds->done) return;
    const bool keep = ds->hn >= 0.70710678118654752 * ds->wnorm;
    if (threadIdx.x == 0) ds->skip2 = keep ? 1 : 0;
    if (keep)
        for (int i = threadIdx.x; i < k; i += blockDim.x) ds->h2[i] = 0.0;
}

__global__ void gmres_gram_step(DevState *ds, int j) {
    if (ds->done) return;
    constexpr int L = kMaxRestart + 1;
    __shared__ double h1[L];
    const int t = threadIdx.x;
    if (t <= j) {
        ds->G[t * L + j] = ds->gcol[t];
        ds->G[j * L + t] = ds->gcol[t];
        h1[t] = ds->h1[t];
    }
    __syncthreads();
    if (t <= j) {
        double gh = 0.0;
        for (int l = 0; l <= j; ++l) gh += ds->G[t * L + l] * h1[l];
        ds->h1[t] = h1[t] + (h1[t] - gh);
        ds->h2[t] = 0.0;
    }
}

__global__ void gmres_backsolve(DevState *ds, int m) {
    const int n = ds->jend;
    for (int i = n - 1; i >= 0; --i) {
        double s = ds->g[i];
        for (int q = i + 1; q < n; ++q) s -= ds->H[i * m + q] * ds->y[q];
        ds->y[i] = s / ds->H[i * m + i];
    }
}

// BiCGSTAB scalar steps (single thread).  red[]: 0 <rh,r>, 1 <rh,v>, 2 ||v||,
// 3 ||s||, 4 <t,s>, 5 <t,t>, 8 ||rh||, 9 ||r||, 10 beta, 11 half-step flag.
__global__ void bicg_beta(DevState *ds, double btol) {
    if (ds->done) return;
    const double rho1 = ds->red[0];
    if (!isfinite(rho1)) return raise_status(ds, RSV_ENAN);
    if (fabs(rho1) <= btol * ds->red[8] * ds->red[9]) return raise_status(ds, RSV_EBREAKDOWN);
    ds->rho1 = rho1;
    ds->red[10] = (rho1 / ds->rho) * (ds->alpha / ds->omega);
}

__global__ void bicg_alpha(DevState *ds, double btol) {
    if (ds->done) return;
    const double rv = ds->red[1];
    if (!isfinite(rv)) return raise_status(ds, RSV_ENAN);
    if (fabs(rv) <= btol * ds->red[8] * ds->red[2]) return raise_status(ds, RSV_EBREAKDOWN);
    ds->alpha = ds->rho1 / rv;
}

__global__ void bicg_check_s(DevState *ds) {
    if (ds->done) return;
    ds->iters += 1;
    const double sn = ds->red[3];
    if (!isfinite(sn)) return raise_status(ds, RSV_ENAN);
    if (sn <= ds->tol) {
        ds->red[11] = 1.0;  // x += alpha ph pending
        ds->done = 1;
    }
}

__global__ void bicg_omega(DevState *ds, double btol) {
    if (ds->done) return;
    const double ts = ds->red[4], tt = ds->red[5];
    if (!isfinite(tt)) return raise_status(ds, RSV_ENAN);
    if (!(tt > 0.0)) return raise_status(ds, RSV_EBREAKDOWN);
    const double om = ts / tt;
    if (fabs(om) <= btol) return raise_status(ds, RSV_EBREAKDOWN);
    ds->omega = om;
}

// stall_limit > 0 (FP32 inner solves of refinement): stop when the residual
// has not dropped below 0.99 of its best for stall_limit passes (FP32
// BiCGSTAB can stagnate above the inner tolerance; the FP64 outer step
// continues from the iterate reached).  red[14] best residual, red[15] count.
__global__ void bicg_finish_iter(DevState *ds, int stall_limit) {
    if (ds->done) return;
    ds->rho = ds->rho1;
    const double rn = ds->red[9];
    if (!isfinite(rn)) return raise_status(ds, RSV_ENAN);
    if (rn <= ds->tol || ds->iters >= ds->maxit) {
        ds->done = 1;
        return;
    }
    if (stall_limit > 0) {
        if (rn < 0.99 * ds->red[14]) {
            ds->red[14] = rn;
            ds->red[15] = 0.0;
        } else if ((ds->red[15] += 1.0) >= stall_limit) {
            ds->red[11] = 3.0;  // stopped on stagnation
            ds->done = 1;
        }
    }
}

__global__ void bicg_init(DevState *ds) {
    ds->rho = ds->alpha = ds->omega = 1.0;
    ds->red[8] = ds->red[9];
    ds->red[11] = 0.0;
    ds->red[14] = ds->red[9];
    ds->red[15] = 0.0;
    ds->done = 0;
}

// p = r + beta (p - omega v)
template <typename T>
__global__ void bicg_update_p(int64_t n, const DevState *ds, const T *r, const T *v, T *p) {
    if (ds->done) return;
    const T beta = (T)ds->red[10], om = (T)ds->omega;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        p[i] = r[i] + beta * (p[i] - om * v[i]);
}

// s = r - alpha v
template <typename T>
__global__ void bicg_update_s(int64_t n, const DevState *ds, const T *r, const T *v, T *s) {
    if (ds->done) return;
    const T al = (T)ds->alpha;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) s[i] = r[i] - al * v[i];
}

// x += alpha ph when the half step converged
template <typename T>
__global__ void bicg_half_x(int64_t n, DevState *ds, const T *ph, T *x) {
    if (ds->red[11] != 1.0) return;
    const T al = (T)ds->alpha;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) x[i] += al * ph[i];
}

__global__ void bicg_consume_half(DevState *ds) {
    if (ds->red[11] == 1.0) ds->red[11] = 2.0;
}

// x += alpha ph + omega sh; r = s - omega t
template <typename T>
__global__ void bicg_update_xr(int64_t n, const DevState *ds, const T *ph, const T *sh, const T *s, const T *t,
                               T *x, T *r) {
    if (ds->done) return;
    const T al = (T)ds->alpha, om = (T)ds->omega;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        x[i] += al * ph[i] + om * sh[i];
        r[i] = s[i] - om * t[i];
    }
}

int egrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace
}  // namespace rsv

using namespace rsv;

namespace {

struct HostState {
    double beta;
    int done, status, iters, jend, conv;
};

rsv_status fetch(rsv_solver *s, HostState *h) {
    DevState *ds = s->ds;
    RSV_CUDA_TRY(cudaMemcpyAsync(&h->beta, &ds->beta, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&h->done, &ds->done, 5 * sizeof(int), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

rsv_status set_tol(rsv_solver *s, double tol) {
    RSV_CUDA_TRY(cudaMemcpyAsync(&s->ds->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, s->st));
    return RSV_OK;
}

// Restarted GMRES(m) / FGMRES on A x = b in precision T, from the x given,
// until ||b - A x|| <= tol or the device iteration counter reaches p.maxit.
// confirm: a cycle whose residual estimate meets tol is confirmed on the
// residual recomputed in T (FP64 solves).  The FP32 inner solves of
// iterative refinement stop on the estimate instead: an FP32 recomputed
// residual has a rounding floor that can sit above the inner tolerance, and
// the FP64 outer residual checks the correction anyway.  Counts cycles.
template <typename T>
rsv_status gmres_run(rsv_solver *s, const T *b, T *x, double tol, int *cycles, bool confirm) {
    const int64_t n = s->n, ldv = s->ldv;
    const int m = s->p.restart;
    const bool flex = s->p.solver == RSV_FGMRES;
    // FP32 GMRES orthogonalises with delayed reorthogonalisation (gmres_dcgs2_step): the
    // preconditioner runs on the not yet reorthogonalised u_j, which a flexible method
    // would have to correct in Z as well, so FGMRES keeps the two explicit passes.
    const bool delayed = !flex && sizeof(T) == 4;
    // FP64 GMRES keeps z_j = M^{-1} v_j of every step and updates x += Z y, with no application
    // of the preconditioner per restart (as FGMRES does).  FP32 forms M^{-1} (V y) instead:
    // V is orthonormal, so V y has no cancellation, while an FP32 sum of the z_j can cancel;
    // with the Z form the FP32 inner counts moved far from the oracle's refinement model
    // (GMRES + block Jacobi on 33x17x9: 1008 against 1231).
    const bool zupdate = flex || sizeof(T) == 8;
    DevState *ds = s->ds;
    T *V = (T *)s->kw.V, *Z = (T *)s->kw.Z, *w = (T *)s->kw.w, *t = (T *)s->kw.t;
    HostState h{};
    RSV_TRY(set_tol(s, tol));
    for (;;) {
        RSV_CUDA_TRY(residual<T>(s, b, x, V, &ds->beta));
        RSV_TRY(fetch(s, &h));
        if (h.status != RSV_OK) return (rsv_status)h.status;
        if (!std::isfinite(h.beta)) return RSV_ENAN;
        if (h.beta <= tol) return RSV_OK;
        if (h.iters >= s->p.maxit) return RSV_ENOCONV;
        ++*cycles;
        rsv::count_launches(1);
        gmres_cycle_init<<<1, 1, 0, s->st>>>(ds);
        if (!delayed) RSV_CUDA_TRY(launch_scale_inv<T>(s->st, n, V, &ds->beta, nullptr));  // else u_0 = r
        for (int j = 0; j < m; ++j) {
            T *vj = V + (size_t)j * ldv;
            T *wj = V + (size_t)(j + 1) * ldv;
            T *z = zupdate ? Z + (size_t)j * ldv : t;
            RSV_CUDA_TRY(pc_apply<T>(s, vj, z, &ds->done));
            RSV_CUDA_TRY(spmv<T>(s, T(1), z, T(0), wj, &ds->done));
            if (delayed) {
                // slot j holds u_j, slot j+1 w = A M^{-1} u_j: projections of both in one read
                // of the basis, the step's scalars, then v_j and u_{j+1} in one more read
                RSV_CUDA_TRY(launch_mdot2<T>(s->st, n, wj, vj, V, ldv, j + 1, s->partial, ds->ow, ds->ou,
                                             &ds->counter[0], &ds->done));
                rsv::count_launches(1);
                RSV_CUDA_TRY(launch_pdl(gmres_dcgs2_step, dim3(1), dim3(128), 0, s->st, ds, j, m, 0));
                RSV_CUDA_TRY(launch_dcgs2_update<T>(s->st, n, vj, wj, V, ldv, j, ds->cA, ds->cB, ds->cS, &ds->done));
                continue;
            }
            if (sizeof(T) == 8) {
                // FP64: projections onto V and the Gram matrix's new column in one read of the
                // basis, the second pass's projections from the Gram matrix, then one update
                // w -= V h that also forms ||w||.  The update's own rounding (~1e-16) is far
                // below what the second pass removes, so this is CGS2 with two reads of V.
                RSV_CUDA_TRY(launch_mdot2<T>(s->st, n, wj, vj, V, ldv, j + 1, s->partial, ds->h1, ds->gcol,
                                             &ds->counter[0], &ds->done));
                rsv::count_launches(1);
                gmres_gram_step<<<1, kMaxRestart + 1, 0, s->st>>>(ds, j);
                RSV_CUDA_TRY(launch_maxpy<T>(s->st, n, wj, V, ldv, j + 1, ds->h1, -1.0, wj, s->partial, &ds->hn,
                                             &ds->counter[1], &ds->done));
            } else {
                // FP32: the second pass recomputes the projections of the updated vector, which
                // also removes the first update's FP32 rounding (the Gram-matrix form leaves it,
                // and the inner solves then take about 10% more iterations); it runs when the
                // first pass cancelled more than 1 - 1/sqrt(2) of the norm ("twice is enough")
                RSV_CUDA_TRY(launch_mdot<T>(s->st, n, wj, V, ldv, j + 1, s->partial, ds->h1, &ds->counter[0],
                                            &ds->done, &ds->wnorm));
                if (j + 1 <= kFuseMax<T>) {
                    // the first pass's update also forms the second pass's projections
                    RSV_CUDA_TRY(launch_maxpy_mdot<T>(s->st, n, wj, V, ldv, j + 1, ds->h1, s->partial, ds->h2,
                                                      &ds->hn, &ds->counter[1], &ds->done));
                    rsv::count_launches(1);
                    gmres_reorth_check<<<1, 32, 0, s->st>>>(ds, j + 1);
                } else {
                    RSV_CUDA_TRY(launch_maxpy<T>(s->st, n, wj, V, ldv, j + 1, ds->h1, -1.0, wj, s->partial, &ds->hn,
                                                 &ds->counter[1], &ds->done));
                    rsv::count_launches(1);
                    gmres_reorth_check<<<1, 32, 0, s->st>>>(ds, j + 1);
                    RSV_CUDA_TRY(launch_mdot<T>(s->st, n, wj, V, ldv, j + 1, s->partial, ds->h2, &ds->counter[0],
                                                &ds->done, nullptr, &ds->skip2));
                }
                RSV_CUDA_TRY(launch_maxpy<T>(s->st, n, wj, V, ldv, j + 1, ds->h2, -1.0, wj, s->partial, &ds->hn,
                                             &ds->counter[1], &ds->done, &ds->skip2));
            }
            rsv::count_launches(1);
            gmres_givens<<<1, kMaxRestart, 0, s->st>>>(ds, j, m);
            if (s->pc_type == RSV_PC_CPR_LEARNED) RSV_CUDA_TRY(learned_watch(s, j));
            RSV_CUDA_TRY(launch_scale_inv<T>(s->st, n, wj, &ds->hn, &ds->done));
        }
        if (delayed) {
            // the cycle's last column waits for u_m's reorthogonalisation: <u_m, V_i> and <u_m, u_m>
            RSV_CUDA_TRY(launch_mdot<T>(s->st, n, V + (size_t)m * ldv, V, ldv, m, s->partial, ds->ou,
                                        &ds->counter[0], &ds->done, &ds->wnorm));
            rsv::count_launches(1);
            gmres_dcgs2_step<<<1, 128, 0, s->st>>>(ds, m, m, 1);
        }
        RSV_TRY(fetch(s, &h));
        if (h.status != RSV_OK && h.status != RSV_EBREAKDOWN) return (rsv_status)h.status;
        if (h.jend > 0) {
            rsv::count_launches(1);
            gmres_backsolve<<<1, 1, 0, s->st>>>(ds, m);
            if (zupdate) {
                RSV_CUDA_TRY(launch_maxpy<T>(s->st, n, x, Z, ldv, h.jend, ds->y, 1.0, x, s->partial, nullptr,
                                             &ds->counter[1], nullptr));
            } else {
                RSV_CUDA_TRY(launch_maxpy<T>(s->st, n, (const T *)nullptr, V, ldv, h.jend, ds->y, 1.0, w, s->partial,
                                             nullptr, &ds->counter[1], nullptr));
                RSV_CUDA_TRY(pc_apply<T>(s, w, t, nullptr));
                RSV_CUDA_TRY(launch_axpby<T>(s->st, n, T(1), t, T(1), x, x));
            }
        }
        if (h.status == RSV_EBREAKDOWN) return RSV_EBREAKDOWN;
        if (!confirm && h.conv) return RSV_OK;
    }
}

// Right-preconditioned BiCGSTAB in precision T from the x given.
template <typename T>
rsv_status bicgstab_run(rsv_solver *s, const T *b, T *x, double tol) {
    const int64_t n = s->n, ldv = s->ldv;
    DevState *ds = s->ds;
    T *r = (T *)s->kw.V, *rh = r + ldv, *p = r + 2 * ldv, *v = r + 3 * ldv, *ph = r + 4 * ldv, *sh = r + 5 * ldv,
      *sv = r + 6 * ldv, *t = r + 7 * ldv;  // s (sv) and t adjacent: one two-column dot
    const double btol = s->p.btol;
    RSV_TRY(set_tol(s, tol));
    RSV_CUDA_TRY(residual<T>(s, b, x, r, &ds->red[9]));
    RSV_CUDA_TRY(cudaMemcpyAsync(rh, r, sizeof(T) * n, cudaMemcpyDeviceToDevice, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(T) * n, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(T) * n, s->st));
    rsv::count_launches(1);
    bicg_init<<<1, 1, 0, s->st>>>(ds);
    double rn0 = 0.0;
    int status0 = 0;
    RSV_CUDA_TRY(cudaMemcpyAsync(&rn0, &ds->red[9], sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&status0, &ds->status, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    if (status0 != RSV_OK) return (rsv_status)status0;  // a device-side failure (e.g. a timed-out wait) first
    if (!std::isfinite(rn0)) return RSV_ENAN;
    if (rn0 <= tol) return RSV_OK;
    const int g = egrid(n);
    const int kBatch = 8;
    HostState h{};
    for (;;) {
        for (int it = 0; it < kBatch; ++it) {
            const int *done = &ds->done;
            RSV_CUDA_TRY(launch_dot<T>(s->st, n, rh, r, s->partial, &ds->red[0], &ds->counter[0], 0, done));
            rsv::count_launches(2);
            bicg_beta<<<1, 1, 0, s->st>>>(ds, btol);
            bicg_update_p<T><<<g, 256, 0, s->st>>>(n, ds, r, v, p);
            RSV_CUDA_TRY(pc_apply<T>(s, p, ph, done));
            RSV_CUDA_TRY(spmv<T>(s, T(1), ph, T(0), v, done));
            RSV_CUDA_TRY(launch_dot<T>(s->st, n, rh, v, s->partial, &ds->red[1], &ds->counter[0], 0, done));
            RSV_CUDA_TRY(launch_dot<T>(s->st, n, v, v, s->partial, &ds->red[2], &ds->counter[0], 1, done));
            rsv::count_launches(2);
            bicg_alpha<<<1, 1, 0, s->st>>>(ds, btol);
            bicg_update_s<T><<<g, 256, 0, s->st>>>(n, ds, r, v, sv);
            RSV_CUDA_TRY(launch_dot<T>(s->st, n, sv, sv, s->partial, &ds->red[3], &ds->counter[0], 1, done));
            rsv::count_launches(3);
            bicg_check_s<<<1, 1, 0, s->st>>>(ds);
            bicg_half_x<T><<<g, 256, 0, s->st>>>(n, ds, ph, x);
            bicg_consume_half<<<1, 1, 0, s->st>>>(ds);
            RSV_CUDA_TRY(pc_apply<T>(s, sv, sh, done));
            RSV_CUDA_TRY(spmv<T>(s, T(1), sh, T(0), t, done));
            RSV_CUDA_TRY(launch_mdot<T>(s->st, n, t, sv, ldv, 2, s->partial, &ds->red[4], &ds->counter[0], done));
            rsv::count_launches(2);
            bicg_omega<<<1, 1, 0, s->st>>>(ds, btol);
            bicg_update_xr<T><<<g, 256, 0, s->st>>>(n, ds, ph, sh, sv, t, x, r);
            RSV_CUDA_TRY(launch_dot<T>(s->st, n, r, r, s->partial, &ds->red[9], &ds->counter[0], 1, done));
            rsv::count_launches(1);
            bicg_finish_iter<<<1, 1, 0, s->st>>>(ds, sizeof(T) == 4 ? 30 : 0);
        }
        RSV_CUDA_TRY(cudaGetLastError());
        RSV_TRY(fetch(s, &h));
        if (h.done || h.status != RSV_OK) break;
    }
    if (h.status != RSV_OK) return (rsv_status)h.status;
    double rn = 0.0, half = 0.0;
    RSV_CUDA_TRY(cudaMemcpyAsync(&rn, &ds->red[9], sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&half, &ds->red[11], sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    if (half == 1.0 || half == 2.0 || rn <= tol) return RSV_OK;
    if (half == 3.0) return RSV_ENOCONV;  // stagnated: the refinement loop carries on
    return RSV_ENOCONV;
}

// FP64 solve: the Krylov method runs directly on the FP64 system.
rsv_status solve_fp64(rsv_solver *s, const double *b, double *x, double tol, rsv_solve_info *info) {
    int cycles = 0;
    rsv_status st = (s->p.solver == RSV_BICGSTAB) ? bicgstab_run<double>(s, b, x, tol)
                                                   : gmres_run<double>(s, b, x, tol, &cycles, true);
    info->restarts = cycles;
    return st;
}

// Mixed precision: FP64 iterative refinement around FP32 inner solves.
rsv_status solve_mixed(rsv_solver *s, const double *b, double *x, double tol, rsv_solve_info *info) {
    const int64_t n = s->n;
    DevState *ds = s->ds;
    int cycles = 0, outer = 0;
    rsv_status result = RSV_ENOCONV;
    for (;;) {
        RSV_CUDA_TRY(residual<double>(s, b, x, s->r64, &ds->red[13]));
        double rn = 0.0;
        int iters = 0, status = 0;
        RSV_CUDA_TRY(cudaMemcpyAsync(&rn, &ds->red[13], sizeof(double), cudaMemcpyDeviceToHost, s->st));
        RSV_CUDA_TRY(cudaMemcpyAsync(&status, &ds->status, sizeof(int), cudaMemcpyDeviceToHost, s->st));
        RSV_CUDA_TRY(cudaMemcpyAsync(&iters, &ds->iters, sizeof(int), cudaMemcpyDeviceToHost, s->st));
        RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
        if (status != RSV_OK) { result = (rsv_status)status; break; }
        if (!std::isfinite(rn)) { result = RSV_ENAN; break; }
        if (rn <= tol) { result = RSV_OK; break; }
        if (outer >= s->p.max_outer || iters >= s->p.maxit) { result = RSV_ENOCONV; break; }
        ++outer;
        RSV_CUDA_TRY(launch_to_f32_scaled(s->st, n, s->r64, &ds->red[13], s->rf));
        RSV_CUDA_TRY(cudaMemsetAsync(s->df, 0, sizeof(float) * n, s->st));
        // inner tolerance relative to ||r||: inner_rtol, or less strict on the last step, which
        // only needs to bring ||r|| below tol (factor 2 of margin)
        const double itol = std::max(s->p.inner_rtol, 0.5 * tol / rn);
        rsv_status ist = (s->p.solver == RSV_BICGSTAB) ? bicgstab_run<float>(s, s->rf, s->df, itol)
                                                        : gmres_run<float>(s, s->rf, s->df, itol, &cycles, false);
        if (ist != RSV_OK && ist != RSV_ENOCONV && ist != RSV_EBREAKDOWN) { result = ist; break; }
        if (ist == RSV_EBREAKDOWN) {
            // a breakdown of the inner solve still leaves a usable correction;
            // clear the device flag so that the outer loop can continue
            RSV_CUDA_TRY(cudaMemsetAsync(&ds->status, 0, sizeof(int), s->st));
        }
        RSV_CUDA_TRY(launch_add_f32_scaled(s->st, n, s->df, &ds->red[13], x));
    }
    info->restarts = cycles;
    info->outer_iters = outer;
    return result;
}

void solver_free(rsv_solver *s) {
    if (!s) return;
    cudaStreamSynchronize(s->st);
    for (void *p : {(void *)s->ds, (void *)s->partial, s->kw.V, s->kw.Z, s->kw.w, s->kw.t, (void *)s->r64,
                    (void *)s->d_b, (void *)s->d_x, (void *)s->rf, (void *)s->df, (void *)s->dinv,
                    (void *)s->dinv32, (void *)s->acc})
        if (p) cudaFree(p);
    free_schedule(&s->sch);
    free_tiles(&s->tiles);
    free_cpr(&s->cpr);
    free_batch(s);
    learned_free(s);
    if (s->e0) cudaEventDestroy(s->e0);
    if (s->e1) cudaEventDestroy(s->e1);
    delete s;
}

rsv_status read_status(rsv_solver *s, int *status) {
    RSV_CUDA_TRY(cudaMemcpyAsync(status, &s->ds->status, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

}  // namespace

extern "C" {

rsv_status rsv_solver_create(rsv_mat *A, const rsv_solver_params *p, rsv_solver **out) {
    if (!A || !p || !out) return RSV_EINVAL;
    if (p->solver < RSV_GMRES || p->solver > RSV_FGMRES) return RSV_EINVAL;
    if (p->restart < 1 || p->restart > kMaxRestart || p->maxit < 0 || !(p->rtol >= 0.0) || !(p->atol >= 0.0) ||
        !(p->btol >= 0.0) || p->watchdog < 1)
        return RSV_EINVAL;
    if (p->precision != RSV_PREC_FP64 && p->precision != RSV_PREC_MIXED) return RSV_EINVAL;
    if (p->precision == RSV_PREC_MIXED && (!(p->inner_rtol > 0.0) || !(p->inner_rtol < 1.0) || p->max_outer < 1))
        return RSV_EINVAL;
    if (p->precision == RSV_PREC_MIXED && !A->d_v32) return RSV_EINVAL;  // matrix created without an FP32 copy
    rsv_solver *s = new (std::nothrow) rsv_solver();
    if (!s) return RSV_ENOMEM;
    s->A = A;
    s->p = *p;
    s->st = A->stream;
    s->n = 3 * A->nb;
    s->ldv = (s->n + 3) & ~int64_t(3);
    s->mixed = p->precision == RSV_PREC_MIXED;
    const int64_t n = std::max<int64_t>(s->ldv, 4);
    const int m = p->restart;
    const size_t es = s->mixed ? sizeof(float) : sizeof(double);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
    };
    alloc((void **)&s->ds, sizeof(DevState));
    alloc((void **)&s->partial, sizeof(double) * 2 * (kMaxRestart + 16) * kRedBlocks);
    if (p->solver == RSV_BICGSTAB) {
        alloc(&s->kw.V, 8 * n * es);
    } else {
        alloc(&s->kw.V, (size_t)(m + 1) * n * es);
        // M^{-1} of every basis vector: FGMRES, and FP64 GMRES (its update from them needs no apply per restart)
        if (p->solver == RSV_FGMRES || !s->mixed) alloc(&s->kw.Z, (size_t)m * n * es);
    }
    alloc(&s->kw.w, n * es);
    alloc(&s->kw.t, n * es);
    alloc((void **)&s->r64, n * sizeof(double));
    alloc((void **)&s->d_b, n * sizeof(double));
    alloc((void **)&s->d_x, n * sizeof(double));
    if (s->mixed) {
        alloc((void **)&s->rf, n * sizeof(float));
        alloc((void **)&s->df, n * sizeof(float));
    }
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

rsv_status rsv_precond_setup(rsv_solver *s, int pc_type, const rsv_pc_params *params) {
    if (!s || pc_type < RSV_PC_NONE || pc_type > RSV_PC_CPR_FFPF) return RSV_EINVAL;
    if (pc_type == RSV_PC_CPR_LEARNED && (s->mixed || s->p.solver != RSV_FGMRES)) return RSV_ENOTSUP;
    if (pc_type == RSV_PC_CPR_LEARNED && !s->unet) return RSV_EINVAL;
    const bool cpr = is_cpr_type(pc_type);
    rsv_pc_params pcp;
    rsv_pc_params_default(&pcp);
    if (params) pcp = *params;
    if (pcp.gmg_max_levels < 1 || pcp.gmg_max_levels > kMaxLevels || pcp.gmg_max_coarse < 1 ||
        pcp.gmg_max_coarse > 1024 || pcp.gmg_sweeps < 0 || pcp.gmg_sweeps > 16 || pcp.decoupling < 0 ||
        pcp.decoupling > 2 || pcp.coarsening < 0 || pcp.coarsening > 1)
        return RSV_EINVAL;
    if (cpr && pcp.decoupling == 2 && !s->acc) return RSV_EINVAL;  // true-IMPES needs the accumulation blocks
    rsv_mat *A = s->A;
    s->pc_type = -1;
    RSV_CUDA_TRY(cudaEventRecord(s->e0, s->st));
    RSV_CUDA_TRY(cudaMemsetAsync(&s->ds->status, 0, sizeof(int), s->st));
    if (pc_type != RSV_PC_NONE && !s->dinv)
        RSV_CUDA_TRY(cudaMalloc((void **)&s->dinv, sizeof(double) * 9 * std::max<int64_t>(A->nb, 1)));
    if (pc_type == RSV_PC_BJACOBI) {
        if (s->mixed && !s->dinv32)
            RSV_CUDA_TRY(cudaMalloc((void **)&s->dinv32, sizeof(float) * 9 * std::max<int64_t>(A->nb, 1)));
        RSV_CUDA_TRY(launch_bj_setup(A, s->mixed, s->dinv, s->mixed ? s->dinv32 : nullptr, &s->ds->status));
    }
    if (pc_type == RSV_PC_BILU0 || cpr) {
        if (!s->sch.cells) RSV_CUDA_TRY(build_schedule(A, &s->sch));
        RSV_CUDA_TRY(launch_ilu_setup(A, s->sch, s->mixed, s->dinv, &s->ds->status));
        if (s->mixed)
            RSV_CUDA_TRY(tiles_setup<float>(A, s->dinv, &s->tiles));
        else
            RSV_CUDA_TRY(tiles_setup<double>(A, s->dinv, &s->tiles));
    }
    if (cpr && A->nsys > 1) return RSV_ENOTSUP;
    if (cpr)
        RSV_CUDA_TRY(cpr_setup(A, s->mixed, pcp.gmg_max_levels, pcp.gmg_max_coarse, pcp.gmg_sweeps, pcp.decoupling,
                               s->acc, pcp.coarsening, &s->cpr, &s->ds->status));
    if (cpr && pcp.coarsening == 1) {
        int status0 = 0;
        RSV_TRY(read_status(s, &status0));  // the decoupling's pivots first
        if (status0 != RSV_OK) return (rsv_status)status0;
        RSV_TRY(amg_setup(A, &s->cpr, pcp.gmg_max_levels, pcp.gmg_max_coarse, pcp.gmg_sweeps));
    }
    RSV_CUDA_TRY(cudaEventRecord(s->e1, s->st));
    int status = 0;
    RSV_TRY(read_status(s, &status));
    float ms = 0.f;
    RSV_CUDA_TRY(cudaEventElapsedTime(&ms, s->e0, s->e1));
    s->ms_setup = ms;
    if (status != RSV_OK) return (rsv_status)status;
    s->pc_type = pc_type;
    s->pcp = pcp;
    s->pc_version = A->version;
    return RSV_OK;
}

static rsv_status pc_check(rsv_solver *s, const void *r, const void *z) {
    if (!s || !r || !z || r == z) return RSV_EINVAL;
    if (s->pc_type < 0 || s->pc_version != s->A->version) return RSV_EINVAL;
    return RSV_OK;
}

rsv_status rsv_precond_set_accumulation(rsv_solver *s, const double *acc, int on_device) {
    if (!s) return RSV_EINVAL;
    if (!acc) {
        if (s->acc) {
            RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
            cudaFree(s->acc);
            s->acc = nullptr;
        }
        return RSV_OK;
    }
    const size_t bytes = sizeof(double) * 9 * (size_t)std::max<int64_t>(s->A->nb, 1);
    if (!s->acc) RSV_CUDA_TRY(cudaMalloc((void **)&s->acc, bytes));
    RSV_CUDA_TRY(cudaMemcpyAsync(s->acc, acc, sizeof(double) * 9 * (size_t)s->A->nb,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

rsv_status rsv_precond_apply(rsv_solver *s, const double *r, double *z) {
    RSV_TRY(pc_check(s, r, z));
    if (s->mixed) return RSV_EINVAL;
    RSV_CUDA_TRY(pc_apply<double>(s, r, z, nullptr));
    return RSV_OK;
}

rsv_status rsv_precond_apply_f32(rsv_solver *s, const float *r, float *z) {
    RSV_TRY(pc_check(s, r, z));
    if (!s->mixed) return RSV_EINVAL;
    RSV_CUDA_TRY(pc_apply<float>(s, r, z, nullptr));
    return RSV_OK;
}

rsv_status rsv_cpr_info(rsv_solver *s, int *nlev, int *dims, double *w_host, double *a7_host) {
    if (!s || !is_cpr_type(s->pc_type)) return RSV_EINVAL;
    const Cpr &P = s->cpr;
    if (nlev) *nlev = P.nlev;
    if (dims)
        for (int l = 0; l < P.nlev; ++l)
            for (int d = 0; d < 3; ++d) dims[3 * l + d] = P.dims[l][d];
    const int64_t nb = s->A->nb;
    if (w_host) RSV_CUDA_TRY(cudaMemcpyAsync(w_host, P.w64, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, s->st));
    if (a7_host) {
        // level stencils, concatenated, each converted from slot-major [7][n] to [n][7]
        std::vector<double> buf;
        int64_t off = 0;
        for (int l = 0; l < P.nlev; ++l) {
            const int64_t n = (int64_t)P.dims[l][0] * P.dims[l][1] * P.dims[l][2];
            buf.resize(7 * n);
            RSV_CUDA_TRY(cudaMemcpyAsync(buf.data(), P.a7[l], sizeof(double) * 7 * n, cudaMemcpyDeviceToHost, s->st));
            RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
            for (int64_t c = 0; c < n; ++c)
                for (int q = 0; q < 7; ++q) a7_host[off + 7 * c + q] = buf[(size_t)q * n + c];
            off += 7 * n;
        }
    }
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

rsv_status rsv_amg_info(rsv_solver *s, int *nlev, int64_t *sizes) {
    if (!s || !is_cpr_type(s->pc_type) || !s->cpr.amg) return RSV_EINVAL;
    return amg_info(s->cpr, nlev, sizes);
}

rsv_status rsv_cpr_vcycle(rsv_solver *s, const double *b, double *x) {
    if (!s || !b || !x || b == x || !is_cpr_type(s->pc_type) || s->mixed)
        return RSV_EINVAL;
    RSV_CUDA_TRY(cpr_vcycle<double>(s->A, s->cpr, b, x));
    return RSV_OK;
}

rsv_status rsv_precond_get_dinv(rsv_solver *s, double *dinv_host) {
    if (!s || !dinv_host || !s->dinv || s->pc_type == RSV_PC_NONE || s->pc_type < 0) return RSV_EINVAL;
    RSV_CUDA_TRY(cudaMemcpyAsync(dinv_host, s->dinv, sizeof(double) * 9 * s->A->nb, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    return RSV_OK;
}

rsv_status rsv_solve(rsv_solver *s, const rsv_vec *b, rsv_vec *x, rsv_solve_info *info) {
    if (!s || !b || !x) return RSV_EINVAL;
    if (b->prec != RSV_PREC_FP64 || x->prec != RSV_PREC_FP64 || b->n != s->n || x->n != s->n) return RSV_EINVAL;
    if (b->data == x->data && s->n > 0) return RSV_EINVAL;
    return rsv_solve_ptr(s, (const double *)b->data, (double *)x->data, 1, info);
}

rsv_status rsv_solve_ptr(rsv_solver *s, const double *b, double *x, int on_device, rsv_solve_info *info) {
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
    RSV_CUDA_TRY(cudaMemsetAsync(s->ds, 0, sizeof(DevState), s->st));
    double bnorm = 0.0;
    RSV_CUDA_TRY(launch_dot<double>(s->st, n, db, db, s->partial, &s->ds->bnorm, &s->ds->counter[0], 1, nullptr));
    RSV_CUDA_TRY(cudaMemcpyAsync(&bnorm, &s->ds->bnorm, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    if (!std::isfinite(bnorm)) return RSV_ENAN;
    const double tol = std::max(s->p.rtol * bnorm, s->p.atol);
    const int maxit = s->p.maxit;
    RSV_CUDA_TRY(cudaMemcpyAsync(&s->ds->maxit, &maxit, sizeof(int), cudaMemcpyHostToDevice, s->st));
    const bool learned = s->pc_type == RSV_PC_CPR_LEARNED;
    if (learned) RSV_TRY(learned_reset(s));
    rsv_solve_info local{};
    rsv_status st = s->mixed ? solve_mixed(s, db, dx, tol, &local) : solve_fp64(s, db, dx, tol, &local);
    if (st == RSV_ECUDA || st == RSV_ENOMEM) return st;
    int fallback_iter = -1;
    if (learned) {
        const rsv_status ls = learned_finish(s, &fallback_iter);
        if (ls != RSV_OK) st = ls;
    }
    // FP64 true residual, recomputed; the iteration count from the device
    double rn = 0.0;
    int iters = 0;
    RSV_CUDA_TRY(residual<double>(s, db, dx, s->r64, &s->ds->red[12]));
    RSV_CUDA_TRY(cudaMemcpyAsync(&rn, &s->ds->red[12], sizeof(double), cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaMemcpyAsync(&iters, &s->ds->iters, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    if (!on_device) RSV_CUDA_TRY(cudaMemcpyAsync(x, s->d_x, sizeof(double) * n, cudaMemcpyDeviceToHost, s->st));
    RSV_CUDA_TRY(cudaEventRecord(s->e1, s->st));
    RSV_CUDA_TRY(cudaStreamSynchronize(s->st));
    float ms = 0.f;
    RSV_CUDA_TRY(cudaEventElapsedTime(&ms, s->e0, s->e1));
    if (info) {
        info->iters = iters;
        info->restarts = local.restarts;
        info->outer_iters = local.outer_iters;
        info->status = st;
        info->true_relres = bnorm > 0 ? rn / bnorm : rn;
        info->ms_setup = s->ms_setup;
        info->ms_solve = ms;
        info->fallback_iter = fallback_iter;
    }
    return st;
}

}  // extern "C"
