/*
 * rsv.h - C ABI of the GB300 reservoir linear-solver library (librsv.so).
 *
 * The library solves the Newton linear systems A x = b of a black-oil-like
 * reservoir model on one GPU: A is the 3x3-block Jacobian of a cell-centred
 * structured nx*ny*nz grid with a seven-point two-point-flux stencil.
 * The calls follow the paper's problem statement: a structured grid
 * (Section "Grid"), the map from cells to unknowns (Section "MAP"), a block
 * matrix and vectors (Section "Distributed Matrices" and "Algebraic
 * Operations"), a solver with rtol/atol/btol/maxit/restart (Section
 * "Solvers", SOLVER structure) and a preconditioner with setup/apply/destroy
 * (Section "Preconditioners", SOLVER_PC and PC_TYPE).
 *
 * Conventions for every entry point:
 *  - Return value: an rsv_status; no call aborts, traps or prints.  On an
 *    error nothing is left half-allocated; output arguments are untouched.
 *  - Handles are opaque and own the device memory they allocate.  Host
 *    arrays passed in are copied before the call returns.
 *  - Device pointers are plain CUDA global-memory addresses on the current
 *    device (for example torch.Tensor.data_ptr()); the caller keeps them
 *    alive for the duration of the call.
 *  - A `stream` argument is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  All device work of a handle is issued on the stream it
 *    was created with; calls that return results to the host synchronise it.
 *  - Cell index c = nx*ny*k + nx*j + i (Section "Grid", default bottom-up
 *    index); unknown 3c+e with e = 0 pressure and e = 1, 2 secondary
 *    (point-interleaved: a permutation of the paper's field-major vector x).
 *  - BSR layout: row_ptr int32[nb+1], col_idx int32[nnzb] ascending per row,
 *    values float64[nnzb][3][3] row-major blocks.
 */
#ifndef RSV_H
#define RSV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RSV_API __attribute__((visibility("default")))
#else
#define RSV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RSV_OK = 0,
    RSV_EINVAL = 1,      /* bad argument (null, size, range, wrong state) */
    RSV_ENOMEM = 2,      /* device or host allocation failed */
    RSV_ECUDA = 3,       /* a CUDA runtime call failed */
    RSV_ENOTSUP = 4,     /* combination not supported */
    RSV_ESINGULAR = 5,   /* a 3x3 pivot or coarse-grid pivot with |p| <= 1e-300 */
    RSV_EBREAKDOWN = 6,  /* Krylov breakdown (rho, <rh,v>, omega or Givens radius vanished) */
    RSV_ENOCONV = 7,     /* maxit reached; x holds the last iterate, info is filled */
    RSV_ETIMEOUT = 8,    /* a bounded device-side wait ran out */
    RSV_ENAN = 9         /* NaN or Inf met in a norm */
} rsv_status;

/* RSV_PC_CPR_LEARNED: CPR whose pressure stage is a trained network (rsv_unet.h)
 * instead of the multigrid V-cycle; FP64 flexible GMRES only.
 * The CPR stage orders (Section "CPR-like preconditioners", Algorithms CPR-FP,
 * CPR-PF, CPR-FPF, CPR-FFPF).  F is the full stage (block ILU(0) of A: restricted
 * additive Schwarz on one subdomain) and P the pressure stage (Pi_p, one GMG
 * V-cycle on A_pp, Pi_r).  The first stage acts on f; every later stage acts on
 * r = f - A x and adds to x:
 *   RSV_PC_CPR      PF    (pressure, then full)
 *   RSV_PC_CPR_FP   FP    (full, then pressure)
 *   RSV_PC_CPR_FPF  FPF   (full, pressure, full)
 *   RSV_PC_CPR_FFPF FFPF  (full, full, pressure, full)
 * All four share one setup (quasi-IMPES weights, GMG hierarchy, ILU(0) factor)
 * and run in FP64 or mixed precision, on single-grid matrices. */
typedef enum {
    RSV_PC_NONE = 0,
    RSV_PC_BJACOBI = 1,
    RSV_PC_BILU0 = 2,
    RSV_PC_CPR = 3,
    RSV_PC_CPR_LEARNED = 4,
    RSV_PC_CPR_FP = 5,
    RSV_PC_CPR_FPF = 6,
    RSV_PC_CPR_FFPF = 7
} rsv_pc_type;
typedef enum { RSV_GMRES = 0, RSV_BICGSTAB = 1, RSV_FGMRES = 2 } rsv_solver_type;
typedef enum { RSV_PREC_FP64 = 0, RSV_PREC_MIXED = 1 } rsv_precision;

typedef struct rsv_grid rsv_grid;
typedef struct rsv_mat rsv_mat;
typedef struct rsv_vec rsv_vec;
typedef struct rsv_solver rsv_solver;

/* Solver parameters (the paper's SOLVER fields rtol, atol, btol, maxit,
 * restart; Section "Solvers").  Convergence: ||b - A x||_2 <=
 * max(rtol ||b||_2, atol), always confirmed on the FP64 true residual.
 * btol: breakdown threshold, relative to the norms involved. */
typedef struct {
    int solver;            /* rsv_solver_type */
    int restart;           /* GMRES restart length m, 1..64 */
    double rtol;
    double atol;
    double btol;
    int maxit;             /* Krylov iterations (Arnoldi steps / BiCGSTAB passes), summed */
    int precision;         /* rsv_precision: FP64, or FP32 inner solves + FP64 refinement */
    double inner_rtol;     /* mixed: inner tolerance relative to the current outer residual */
    int max_outer;         /* mixed: maximum refinement steps */
    long long watchdog;    /* time limit, microseconds, of every bounded device-side wait */
} rsv_solver_params;

/* Preconditioner parameters.  GMG defaults follow the paper's AMG defaults
 * (one V-cycle, at most 6 levels, 2 relaxation sweeps; Section "Algebraic
 * Multigrid Methods", default-parameter figure).  decoupling selects how the CPR
 * orders weight the three equations of a cell into its pressure equation
 * (Section "Numerical experiments" names quasi-IMPES and ABF):
 *   0  quasi-IMPES: w_c = (1, -D01/D11, -D02/D22), D = A_cc (default);
 *   1  ABF: w_c = first row of D^{-1} (each block row premultiplied by D^{-1});
 *      RSV_ESINGULAR at setup when |det D| <= 1e-300;
 *   2  true-IMPES: w_c = first row of C_c^{-1}, C_c the cell's accumulation
 *      block (the time-derivative part of A_cc, given by
 *      rsv_precond_set_accumulation; RSV_EINVAL at setup without it), so that
 *      w_c C_c = (1, 0, 0): the secondary unknowns leave the accumulation terms.
 *      RSV_ESINGULAR at setup when |det C_c| <= 1e-300.
 * The pressure operator is A_pp(c, l) = w_c . A_cl[:, 0] in every case.
 * coarsening selects the pressure stage's hierarchy (Section "Algebraic
 * Multigrid Methods", AMG setup algorithm and V-cycle):
 *   0  geometric: 2x2x2 boxes, Galerkin seven-point levels, red-black
 *      Gauss-Seidel (gmg_sweeps before and after);
 *   1  algebraic: strength threshold 0.5, PMIS coarse points, direct
 *      interpolation, Galerkin products R A P with R = P^T, l1-Jacobi smoothing
 *      (gmg_sweeps before and after), the coarsest level solved exactly.  The
 *      hierarchy is built on the host at rsv_precond_setup from the pressure
 *      operator computed on the device; the V-cycle runs on the device.  Levels:
 *      coarsen while a level has more than gmg_max_coarse points, at most
 *      gmg_max_levels (8 reaches small grids; the paper's default 6 may not),
 *      stopping when a level keeps more than 90% of its points.  RSV_ENOTSUP
 *      when the coarsest level would exceed 1024 points. */
typedef struct {
    int gmg_max_levels;    /* <= 8 */
    int gmg_max_coarse;    /* stop coarsening at or below this many cells */
    int gmg_sweeps;        /* red-black Gauss-Seidel sweeps before and after */
    int decoupling;        /* 0 quasi-IMPES, 1 ABF, 2 true-IMPES */
    int coarsening;        /* pressure hierarchy: 0 geometric (default), 1 algebraic (see below) */
} rsv_pc_params;

/* Filled by rsv_solve. */
typedef struct {
    int iters;             /* Krylov iterations summed over restarts / outer steps */
    int restarts;          /* GMRES cycles */
    int outer_iters;       /* refinement steps (mixed precision), else 0 */
    int status;            /* rsv_status of the solve */
    double true_relres;    /* ||b - A x|| / ||b|| recomputed in FP64 on the device */
    double ms_setup;       /* last rsv_precond_setup, CUDA-event time */
    double ms_solve;       /* this solve, CUDA-event time */
    int fallback_iter;     /* RSV_PC_CPR_LEARNED: iteration at which the solve switched to
                              the plain V-cycle; -1 if it never did (other preconditioners: -1) */
    int pad_;
} rsv_solve_info;

/* Defaults: GMRES, m = 30, rtol 1e-8, atol 0, btol 1e-30, maxit 2000, FP64,
 * inner_rtol 1e-5, max_outer 10, watchdog 2,000,000 us. */
RSV_API void rsv_solver_params_default(rsv_solver_params *p);
/* Defaults: 6 levels, 512 coarse cells, 2 sweeps, quasi-IMPES, geometric coarsening. */
RSV_API void rsv_pc_params_default(rsv_pc_params *p);
RSV_API const char *rsv_status_string(rsv_status s);
/* Text of the last CUDA runtime error seen by a call on this thread that
 * returned RSV_ECUDA or RSV_ENOMEM ("no error" if none). */
RSV_API const char *rsv_last_cuda_error(void);
/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all handles); a diagnostic counter for benchmarks. */
RSV_API uint64_t rsv_kernel_launches(void);

/* ---- grid (Section "Grid": structured grid, default cell index) ---------
 * nx, ny, nz >= 1 and nx*ny*nz*3 < 2^31.  The grid is host-only metadata. */
RSV_API rsv_status rsv_grid_create(int nx, int ny, int nz, rsv_grid **out);
RSV_API void rsv_grid_destroy(rsv_grid *g);

/* ---- matrix (Sections "Distributed Matrices", "Algebraic Operations") ---
 * Creates the seven-point block BSR pattern of the grid on the device (rows
 * ascending, columns ascending: -z, -y, -x, self, +x, +y, +z; the paper's
 * distributed matrix with block size 3 and one process owning every row).
 * Values start at zero.  The grid may be destroyed afterwards.
 * block: unknowns per cell; only 3 is supported (RSV_ENOTSUP otherwise).
 * prec: RSV_PREC_FP64 keeps the FP64 values only (solvers on it must be FP64;
 * saves 36 bytes per block); RSV_PREC_MIXED also keeps an FP32 copy, made at
 * every rsv_mat_set_values, for mixed-precision solvers.  RSV_EINVAL for a
 * null grid/out or another prec.  All device work runs on `stream`. */
RSV_API rsv_status rsv_mat_create_bsr(const rsv_grid *g, int block, int prec, void *stream, rsv_mat **out);
/* Same as rsv_mat_create_bsr(g, 3, RSV_PREC_MIXED, stream, out). */
RSV_API rsv_status rsv_mat_create(const rsv_grid *g, void *stream, rsv_mat **out);
RSV_API void rsv_mat_destroy(rsv_mat *A);
/* A batch of nsys independent grids (dims: int[nsys][3], nx ny nz each) as
 * one block-diagonal matrix: grid s occupies cells [off_s, off_{s+1}) in
 * bottom-up order, unknowns 3*cell + e; values are passed concatenated in
 * the same order.  Solve it with rsv_solve_batched (independent systems) or
 * rsv_solve (the block-diagonal system as a whole).  CPR needs a single grid. */
RSV_API rsv_status rsv_mat_create_batch(int nsys, const int *dims, void *stream, rsv_mat **out);
/* Number of grids and their cell offsets (int64[nsys+1]; either may be NULL). */
RSV_API rsv_status rsv_mat_get_batch(const rsv_mat *A, int *nsys, int64_t *cell_offsets);
/* Host views of the pattern, owned by the matrix (valid until destroy). */
RSV_API rsv_status rsv_mat_get_pattern(const rsv_mat *A, const int32_t **row_ptr, const int32_t **col_idx,
                               int64_t *nb, int64_t *nnzb);
/* Copy nnzb*9 float64 block values (host or device pointer, on_device 0/1)
 * into the matrix.  Invalidates any preconditioner built on it. */
RSV_API rsv_status rsv_mat_set_values(rsv_mat *A, const double *vals, int on_device);

/* y = alpha A x + beta y (Section "Algebraic Operations", first equation).
 * x, y: device float64[3*nb]; x and y must not overlap. */
RSV_API rsv_status rsv_spmv(const rsv_mat *A, double alpha, const double *x, double beta, double *y);
/* Same in FP32: values rounded once to float at set_values time (the copy
 * used by mixed-precision inner solves); x, y device float32[3*nb].
 * RSV_EINVAL on a matrix created with prec RSV_PREC_FP64. */
RSV_API rsv_status rsv_spmv_f32(const rsv_mat *A, float alpha, const float *x, float beta, float *y);

/* ---- vectors (Section "Distributed Matrices": the vector type beside the
 * matrix) ------------------------------------------------------------------
 * A vector is n values of one precision in device memory: float64 for
 * RSV_PREC_FP64, float32 for RSV_PREC_MIXED.
 * rsv_vec_create: owns 3*nx*ny*nz zeroed values (one per unknown of the grid),
 *   allocated with cudaMalloc and zeroed on `stream` (synchronised).
 * rsv_vec_wrap: borrows n values at dev_ptr (device or managed memory, for
 *   example a torch tensor's data_ptr(); aligned to the element size); the
 *   caller keeps the memory alive while the vector is used and frees it
 *   itself.  RSV_EINVAL for a host pointer, a misaligned pointer or n < 0.
 * rsv_vec_set / rsv_vec_get: copy n float64 values in / out (host or device
 *   pointer, on_device 0/1), converting to / from float32 for an FP32 vector,
 *   on `stream`; host copies synchronise it, device copies are stream-ordered.
 * rsv_vec_info: the data pointer, length and precision (any output may be NULL).
 * rsv_vec_destroy frees owned memory only (after the device's work in flight). */
RSV_API rsv_status rsv_vec_create(const rsv_grid *g, int prec, void *stream, rsv_vec **out);
RSV_API rsv_status rsv_vec_wrap(void *dev_ptr, int64_t n, int prec, rsv_vec **out);
RSV_API rsv_status rsv_vec_set(rsv_vec *v, const double *src, int on_device, void *stream);
RSV_API rsv_status rsv_vec_get(const rsv_vec *v, double *dst, int on_device, void *stream);
RSV_API rsv_status rsv_vec_info(const rsv_vec *v, void **dev_ptr, int64_t *n, int *prec);
RSV_API void rsv_vec_destroy(rsv_vec *v);

/* ---- vector algebra (Section "Algebraic Operations") --------------------
 * Device float64 arrays of length n; the scalar result is returned on the
 * host (the call synchronises the stream). */
RSV_API rsv_status rsv_dot(void *stream, int64_t n, const double *x, const double *y, double *result);
RSV_API rsv_status rsv_norm2(void *stream, int64_t n, const double *x, double *result);
/* z = alpha x + beta y (z may alias x or y). */
RSV_API rsv_status rsv_axpby(void *stream, int64_t n, double alpha, const double *x, double beta,
                     const double *y, double *z);

/* Multi-vector dot product that allocates nothing: result[i] = <w, V_i> for
 * i < k, V_i = V + i*ldv (device float64 arrays; result on the host, the call
 * synchronises the stream).  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory when they need a reduction
 * (a device-memory budget already handed out, a callback that forbids
 * allocation, a loop that must not risk an allocator synchronisation).
 * Its reduction scratch is one fixed file-scope device array (about 160 KB,
 * held by every GPU that loads the library until the process exits) instead
 * of memory from the allocator; no call to it allocates or frees.
 * Limits: 1 <= k <= 64 (RSV_EINVAL otherwise), ldv >= n.  Every call ends
 * by synchronising its stream, so it cannot be made while the stream is being
 * captured into a CUDA graph.  The first call on a device resolves the array's
 * device address and keeps it for the life of the process: a cudaDeviceReset
 * in the process invalidates the kept address, so do not call this entry
 * point after resetting a device it has already been called on.
 * Every call reuses the same array, so calls whose GPU work overlaps (other
 * streams, other host threads) race: serialise them. */
RSV_API rsv_status rsv_mdot_noalloc(void *stream, int64_t n, const double *w, const double *V, int64_t ldv, int k,
                                    double *result);

/* ---- solver + preconditioner (Sections "Solvers", "Preconditioners") ----
 * The solver keeps a reference to A (A must outlive it) and allocates its
 * Krylov workspace on A's stream. */
RSV_API rsv_status rsv_solver_create(rsv_mat *A, const rsv_solver_params *p, rsv_solver **out);
RSV_API void rsv_solver_destroy(rsv_solver *s);
/* Build the preconditioner from A's current values:
 *  NONE;  BJACOBI: inverted 3x3 diagonal blocks;
 *  BILU0: block ILU(0) in natural order (Section "Restricted Additive Schwarz
 *         Method": LU x = b <=> L y = b, U x = y; ILU(0) default), scheduled
 *         along i+j+k wavefront hyperplanes;
 *  CPR:   two-stage (Section "CPR-like Preconditioners", CPR-PF): quasi-IMPES
 *         pressure restriction, geometric-multigrid V-cycle on the pressure
 *         matrix (Section "Algebraic Multigrid Methods"), then block ILU(0).
 *  CPR_FP, CPR_FPF, CPR_FFPF: the same stages in the paper's other orders
 *         (see rsv_pc_type).  params->decoupling selects quasi-IMPES or ABF
 *         weights for every CPR type, CPR_LEARNED included (a network trained on
 *         pressure samples of one decoupling expects that decoupling).
 *         RSV_ENOTSUP for a batch matrix (more than one grid).
 * params may be NULL (defaults); RSV_EINVAL for a parameter out of range. */
RSV_API rsv_status rsv_precond_setup(rsv_solver *s, int pc_type, const rsv_pc_params *params);
/* The accumulation blocks C_c of the Jacobian (its time-derivative part; the
 * flux terms excluded), float64[nb][3][3] row-major in cell order, host
 * (on_device = 0) or device (on_device = 1); copied into the solver for the
 * true-IMPES decoupling (rsv_pc_params.decoupling = 2) of later setups.
 * acc = NULL drops them.  Synchronises the solver's stream. */
RSV_API rsv_status rsv_precond_set_accumulation(rsv_solver *s, const double *acc, int on_device);
/* z = M^{-1} r with the current preconditioner of an FP64 solver; device
 * float64[3*nb]; r and z must not overlap.  Returns before the GPU work ends
 * (stream-ordered); a device-side failure surfaces at the next rsv_solve. */
RSV_API rsv_status rsv_precond_apply(rsv_solver *s, const double *r, double *z);
/* Same in FP32 for a mixed-precision solver (its preconditioner is built on
 * the FP32-rounded matrix and stores FP32 factors); device float32[3*nb]. */
RSV_API rsv_status rsv_precond_apply_f32(rsv_solver *s, const float *r, float *z);
/* Inspect a CPR preconditioner of any order (Section "CPR-like Preconditioners"):
 * the number of multigrid levels, their grid dimensions (int[3*nlev]: nx, ny, nz
 * per level, finest first), the decoupling weights (host float64[nb][3]) and
 * the seven-point pressure stencils of every level, finest first,
 * concatenated (host float64[sum_l cells_l][7], slots -z, -y, -x, centre, +x,
 * +y, +z).  Any output may be NULL.  Synchronises the stream. */
RSV_API rsv_status rsv_cpr_info(rsv_solver *s, int *nlev, int *dims, double *w_host, double *a7_host);
/* The algebraic pressure hierarchy of a CPR preconditioner set up with
 * coarsening = 1: its level count and, per level, its points and nonzeros
 * (int64[2 * nlev], finest first; either output may be NULL).  RSV_EINVAL for
 * any other preconditioner. */
RSV_API rsv_status rsv_amg_info(rsv_solver *s, int *nlev, int64_t *sizes);
/* One multigrid V-cycle on the finest pressure system from a zero guess
 * (Section "Algebraic Multigrid Methods", V-cycle algorithm): x = V(b);
 * device float64[nb] (FP64 solver with a CPR preconditioner only). */
RSV_API rsv_status rsv_cpr_vcycle(rsv_solver *s, const double *b, double *x);
/* Copy the inverted diagonal blocks of the preconditioner (block Jacobi:
 * A_ii^{-1}; block ILU(0) and CPR: the ILU factor's U_ii^{-1}) to host
 * float64[nb][3][3]. */
RSV_API rsv_status rsv_precond_get_dinv(rsv_solver *s, double *dinv_host);
/* Solve A x = b (the paper's solve call on a SOLVER with a matrix and two
 * vectors, Section "Solvers").  b, x: FP64 vectors of 3*nb values (RSV_EINVAL
 * for another length or precision, or b and x sharing memory); x holds the
 * initial guess on entry and the solution on return (also on ENOCONV).  The
 * call synchronises the solver's stream; info may be NULL. */
RSV_API rsv_status rsv_solve(rsv_solver *s, const rsv_vec *b, rsv_vec *x, rsv_solve_info *info);
/* The same solve on raw float64[3*nb] arrays, host (on_device = 0: copied in
 * and out inside the call) or device (on_device = 1). */
RSV_API rsv_status rsv_solve_ptr(rsv_solver *s, const double *b, double *x, int on_device, rsv_solve_info *info);

/* Batched solve (the batch extension of the paper's per-process solves; its
 * systems are independent as the paper's subdomain systems are, Section
 * "Grid", partition constraints): every grid of a batch matrix is solved on
 * its own by right-preconditioned BiCGSTAB (solver type must be BICGSTAB,
 * preconditioner NONE, BJACOBI or BILU0), with its own scalars, tolerance
 * rtol * ||b_s||, iteration count and status; FP64 or FP32 inner solves
 * under per-system FP64 refinement.  One pass over all systems is captured
 * in a CUDA graph and replayed.  b, x: FP64 vectors of 3*nb values (the
 * systems' unknowns concatenated), x holds the initial guess; infos:
 * rsv_solve_info[nsys] or NULL.  Returns the first non-OK per-system status,
 * else RSV_OK.  rsv_solve_batched_ptr takes raw float64[3*nb] arrays, host
 * (on_device = 0) or device (on_device = 1). */
RSV_API rsv_status rsv_solve_batched(rsv_solver *s, const rsv_vec *b, rsv_vec *x, rsv_solve_info *infos);
RSV_API rsv_status rsv_solve_batched_ptr(rsv_solver *s, const double *b, double *x, int on_device,
                                         rsv_solve_info *infos);

#ifdef __cplusplus
}
#endif
#endif /* RSV_H */
