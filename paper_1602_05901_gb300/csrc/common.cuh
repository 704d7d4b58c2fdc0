// Internal declarations shared by the CUDA translation units of librsv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rsv.h"

#define RSV_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) {                             \
            rsv::set_last_cuda_error(e_);                    \
            return RSV_ECUDA;                                \
        }                                                    \
    } while (0)

#define RSV_TRY(expr)                                        \
    do {                                                     \
        rsv_status s_ = (expr);                              \
        if (s_ != RSV_OK) return s_;                         \
    } while (0)

namespace rsv {

// Division by an invariant integer as a multiply and a shift (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l for every 0 <= n < 2^31.
// Built on the host for a grid dimension, used by index arithmetic in the kernels.
struct Div32 {
    unsigned m, l;
    static Div32 of(unsigned d) {
        unsigned l = 0;
        while ((1ull << l) < d) ++l;
        return {(unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1), l};
    }
    __device__ __forceinline__ int operator()(int n) const {
        return (int)((__umulhi(m, (unsigned)n) + (unsigned)n) >> l);
    }
};

// Programmatic dependent launch.  A kernel launched by launch_pdl may be scheduled while the
// kernel before it on the stream is still running; it must call pdl_wait() before it touches
// anything that kernel writes (pdl_wait returns once the previous grid has completed and its
// memory is visible; in a kernel launched the ordinary way it returns at once).  pdl_trigger()
// lets the next such kernel be scheduled as soon as every CTA of this grid has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

constexpr int kMaxRestart = 64;
constexpr int kRedBlocks = 304;   // 2 x 152 SMs: grid of every reduction kernel
constexpr int kRedThreads = 256;

void set_last_cuda_error(cudaError_t e);
rsv_status cuda_status(cudaError_t e);
// Process-wide count of kernel launches issued by the library.
void count_launches(uint64_t n);

// Solver scalars that live in device memory so that no Krylov step needs a
// host round trip.  One instance per solver.
struct DevState {
    double H[(kMaxRestart + 1) * kMaxRestart];  // Hessenberg, row-major (m+1) x m, rotated in place
    double cs[kMaxRestart], sn[kMaxRestart];
    double g[kMaxRestart + 1];
    double y[kMaxRestart];
    double h1[kMaxRestart + 1], h2[kMaxRestart + 1];  // CGS2 projection coefficients
    double red[kMaxRestart + 1];                       // generic reduction outputs
    double G[(kMaxRestart + 1) * (kMaxRestart + 1)];   // Gram matrix of the current Arnoldi basis, row-major
    double gcol[kMaxRestart + 1];                      // <v_j, v_i>, i <= j: column j of G
    // delayed CGS2 (FP32 GMRES): projections of the step's two vectors, the unrotated
    // Hessenberg matrix and the update pass's coefficients
    double ow[kMaxRestart + 1], ou[kMaxRestart + 1];
    double Hu[(kMaxRestart + 1) * kMaxRestart];  // row-major (m+1) x m
    double cA[kMaxRestart], cB[kMaxRestart], cS[2];
    double beta, hn, wnorm, tol;
    double rho, rho1, alpha, omega;
    double bnorm;
    int done;       // 1: stop this cycle / iteration loop
    int status;     // rsv_status raised on the device (breakdown, nan, singular)
    int iters;      // Krylov iterations so far (device count)
    int jend;       // Arnoldi steps taken in the current cycle
    int conv;       // the current cycle met the tolerance on its residual estimate
    int skip2;      // the first Gram-Schmidt pass kept enough of the norm: skip the second
    int maxit;
    unsigned counter[4];  // last-block tickets of the reduction kernels
};

struct TileSys {  // one grid of the tile sweeps
    int nx, ny, nz, nTJ, nTK, S, poff, Sp;  // S: steps per tile (Sp: padded to the step group); poff: first position
    int64_t cell0;
};

struct IluTiles {  // packed factor and buffers of the persistent tile sweeps (ilu_tiles.cu)
    int nT = 0, maxS = 0, grid = 0, elem = 0;  // elem: 8 (FP64) or 4 (FP32)
    int64_t rows = 0;         // step rows of all tiles (maxS, rows: padded step counts)
    size_t smem = 0;
    TileSys *tsys = nullptr;  // per grid
    int *tile_sys = nullptr;  // position -> grid
    int64_t *tile_row0 = nullptr;  // position -> first step row
    int2 *order = nullptr;    // tile (J, K) per processing position
    int *pos_of = nullptr;    // grid poff + J * nTK + K -> position
    void *Ff = nullptr;       // forward factor rows  [nT][Sp][32][NQP]
    void *Fb = nullptr;       // backward factor rows [nT][Sp][32][NQP]
    void *Vf = nullptr;       // forward input in tile order [nT][Sp][32][4]
    void *Vb = nullptr;       // backward input (y) in tile order [nT][Sp][32][4]
    void *EJf = nullptr, *EKf = nullptr;  // forward edge hand-off buffers
    void *EJb = nullptr, *EKb = nullptr;  // backward edge hand-off buffers
};

constexpr int kMaxLevels = 8;
struct Cpr {  // CPR pressure stage: quasi-IMPES weights and the GMG hierarchy (cpr.cu)
    bool mixed = false;
    int nlev = 0, sweeps = 2, ncoarse = 0;
    int dims[kMaxLevels][3] = {};
    double *a7[kMaxLevels] = {};  // FP64 seven-point stencils, slot-major [7][n]
    void *a7f[kMaxLevels] = {};   // FP32 copies (mixed precision)
    void *a7s[kMaxLevels] = {};   // colour-split copies in T for the smoother (every level but the coarsest)
    void *x[kMaxLevels] = {}, *b[kMaxLevels] = {};  // per-level solution and right-hand side (T)
    double *w64 = nullptr;        // quasi-IMPES weights [nb][3], FP64
    void *w = nullptr;            // weights in T
    double *dense = nullptr, *minv = nullptr, *work = nullptr;  // coarsest LU / inverse / scratch
    int *piv = nullptr;
    void *r = nullptr, *z = nullptr, *xp = nullptr;  // full-stage residual and ILU correction (T)
    void *apc = nullptr;          // pressure column of every block [nnzb][3] (T): CPR-PF's stage-two residual
    void *amg = nullptr;          // algebraic hierarchy (amg.cu) when the pressure stage coarsens algebraically
};

struct Schedule {  // i+j+k wavefront hyperplanes
    std::vector<int> plane_ptr;  // host, nplanes+1
    int32_t *cells = nullptr;    // device, nb cell indices grouped by plane (ascending within)
    int nplanes = 0;
};

}  // namespace rsv

struct rsv_grid {
    int nx, ny, nz;
};

namespace rsv {
// One structured grid of a (possibly batched) matrix: its dims and first cell.
struct SysGrid {
    int nx, ny, nz, pad;
    int64_t cell0;
};
}  // namespace rsv

struct rsv_mat {
    int nx, ny, nz;                 // dims of the first (for a single-grid matrix: the only) grid
    int nsys = 1;                   // >1: block-diagonal batch of independent grids
    std::vector<rsv::SysGrid> h_sys;
    rsv::SysGrid *d_sys = nullptr;  // per grid
    int32_t *d_sys_of_cell = nullptr;  // grid of each cell
    int spmv_rows64 = 128;          // block rows per CTA of the FP64 SpMV (timed once per matrix)
    int spmv_rows32 = 128;          // the same for the FP32 copy
    bool spmv_tuned = false;
    int64_t nb, nnzb;
    cudaStream_t stream;
    std::vector<int32_t> h_rp, h_ci;
    int32_t *d_rp = nullptr, *d_ci = nullptr;
    double *d_v = nullptr;   // nnzb*9 (+ tail pad)
    float *d_v32 = nullptr;  // FP32 copy of the values (matrices created for mixed precision only)
    uint64_t version = 0;
};

// A vector of the boundary: n values of one precision in device memory, owned
// (rsv_vec_create) or borrowed (rsv_vec_wrap).
struct rsv_vec {
    void *data = nullptr;
    int64_t n = 0;
    int prec = 0;          // RSV_PREC_FP64: double, RSV_PREC_MIXED: float
    bool owned = false;
};

namespace rsv {

// ---- launchers implemented in spmv.cu
// One-time kernel attributes (large dynamic shared memory); called at matrix creation.
cudaError_t spmv_init();
// status (optional): receives RSV_ETIMEOUT when a CTA's staged copies do not arrive within
// timeout_ns; the rows that CTA still owed are then written as NaN.
cudaError_t launch_spmv_f64(const rsv_mat *A, double alpha, const double *x, double beta, double *y,
                            const int *done, int *status = nullptr, unsigned long long timeout_ns = 2000000000ull);
cudaError_t launch_spmv_f32(const rsv_mat *A, float alpha, const float *x, float beta, float *y,
                            const int *done, int *status = nullptr, unsigned long long timeout_ns = 2000000000ull);
cudaError_t launch_cast_f64_f32(cudaStream_t st, int64_t n, const double *a, float *b);
// Time the SpMV's block-rows-per-CTA candidates (32, 64, 128) on A's pattern and keep the
// fastest per precision; once per matrix (later calls return at once).
cudaError_t spmv_autotune(rsv_mat *A);
// r = f - A (p_c, 0, 0)_c from the blocks' pressure columns apc [nnzb][3] (T = double or float).
template <typename T>
cudaError_t launch_pressure_residual(const rsv_mat *A, const T *apc, const T *p, const T *f, T *r, const int *done,
                                     int *status, unsigned long long timeout_ns);

// ---- launchers implemented in blas.cu (T = double or float; reductions in FP64)
// out[i] = <w, V_i> for i < k; V_i = V + i*ldv.  Deterministic two-level reduction.
// self_nrm (optional): also out[k] = <w, w> and *self_nrm = ||w||.  skip (optional): a second
// device flag that, like done, makes the kernel return at once.
template <typename T>
cudaError_t launch_mdot(cudaStream_t st, int64_t n, const T *w, const T *V, int64_t ldv, int k, double *partial,
                        double *out, unsigned *counter, const int *done, double *self_nrm = nullptr,
                        const int *skip = nullptr);
// ow[i] = <w, V_i> and ou[i] = <u, V_i> for i < k (k <= kMaxRestart + 1), one read of the basis;
// partial needs 2 * 8 * ceil(k / 8) slots of kRedBlocks doubles.
template <typename T>
cudaError_t launch_mdot2(cudaStream_t st, int64_t n, const T *w, const T *u, const T *V, int64_t ldv, int k,
                         double *partial, double *ow, double *ou, unsigned *counter, const int *done);
// out = base + sgn * sum_i c[i] V_i (base may be null); if nrm != nullptr, *nrm = ||out||_2.
template <typename T>
cudaError_t launch_maxpy(cudaStream_t st, int64_t n, const T *base, const T *V, int64_t ldv, int k, const double *c,
                         double sgn, T *out, double *partial, double *nrm, unsigned *counter, const int *done,
                         const int *skip = nullptr);
// The update pass of a delayed CGS2 Arnoldi step, both outputs in place and elementwise:
// u = cS[0] u - sum_{i<k} cB[i] V_i and w = cS[0] w - cS[1] u_old - sum_{i<k} cA[i] V_i,
// with u and w outside V_0..V_{k-1}.  One read of the k basis vectors, u and w.
template <typename T>
cudaError_t launch_dcgs2_update(cudaStream_t st, int64_t n, T *u, T *w, const T *V, int64_t ldv, int k,
                                const double *cA, const double *cB, const double *cS, const int *done);
// Classical Gram-Schmidt, the first pass's update fused with the second pass's projections:
// w -= sum_i c[i] V_i (in place, in the vector precision), then proj[i] = <w, V_i> for i < k
// and *nrm = ||w||_2.  Each basis value is read once.  Returns cudaErrorInvalidValue (nothing
// launched) when k > kFuseMax<T>; the caller then runs launch_maxpy and launch_mdot.  The k
// basis values of a row block stay in registers: 32 FP32 float4s, or 16 FP64 double2s.
template <typename T> constexpr int kFuseMax = sizeof(T) == 4 ? 32 : 16;
template <typename T>
cudaError_t launch_maxpy_mdot(cudaStream_t st, int64_t n, T *w, const T *V, int64_t ldv, int k, const double *c,
                              double *partial, double *proj, double *nrm, unsigned *counter, const int *done);
// *out = ||x||_2 (sqrt_out=1) or <x,y>
template <typename T>
cudaError_t launch_dot(cudaStream_t st, int64_t n, const T *x, const T *y, double *partial, double *out,
                       unsigned *counter, int sqrt_out, const int *done);
template <typename T>
cudaError_t launch_axpby(cudaStream_t st, int64_t n, T a, const T *x, T b, const T *y, T *z);
// x *= 1/(*s) (device scalar), skipping when *done
template <typename T>
cudaError_t launch_scale_inv(cudaStream_t st, int64_t n, T *x, const double *s, const int *done);
// xf = (float)(x / *s);  x += (*s) * df
cudaError_t launch_to_f32_scaled(cudaStream_t st, int64_t n, const double *x, const double *s, float *xf);
cudaError_t launch_add_f32_scaled(cudaStream_t st, int64_t n, const float *df, const double *s, double *x);

// ---- launchers implemented in precond.cu
cudaError_t build_schedule(const rsv_mat *A, Schedule *sch);
void free_schedule(Schedule *sch);
// from_f32: factor the FP32-rounded values (mixed precision) instead of the FP64 ones.
cudaError_t launch_bj_setup(const rsv_mat *A, bool from_f32, double *dinv, float *dinv32, int *status);
template <typename T>
cudaError_t launch_bj_apply(cudaStream_t st, int64_t nb, const T *dinv, const T *r, T *z, const int *done);
cudaError_t launch_ilu_setup(const rsv_mat *A, const Schedule &sch, bool from_f32, double *dinv, int *status);

// ---- implemented in cpr.cu
// decoupling: 0 quasi-IMPES, 1 ABF, 2 true-IMPES from the accumulation blocks acc [nb][9] (rsv_pc_params).
// coarsening: 0 geometric hierarchy, 1 algebraic (amg_setup runs afterwards, from P->a7[0]).
cudaError_t cpr_setup(const rsv_mat *A, bool mixed, int max_levels, int max_coarse, int sweeps, int decoupling,
                      const double *acc, int coarsening, Cpr *P, int *status);
// ---- implemented in amg.cu
rsv_status amg_setup(const rsv_mat *A, Cpr *P, int max_levels, int max_coarse, int sweeps);
void amg_free(Cpr *P);
rsv_status amg_info(const Cpr &P, int *nlev, int64_t *sizes);
template <typename T>
cudaError_t amg_vcycle(const Cpr &P, cudaStream_t st, const int *done);
void free_cpr(Cpr *P);
template <typename T>
cudaError_t cpr_apply(const rsv_mat *A, const Cpr &P, const IluTiles &tiles, const T *f, T *x, const int *done,
                      int *status, unsigned long long timeout_ns);
template <typename T>
cudaError_t cpr_restrict(const rsv_mat *A, const Cpr &P, const T *f, const int *done);
// The CPR stage orders: `stages` spells one, 'F' (full: block ILU(0)) or 'P' (pressure:
// Pi_p V-cycle Pi_r) per stage; the first acts on f, every later one on f - A x and adds to x.
template <typename T>
cudaError_t cpr_apply_order(const rsv_mat *A, const Cpr &P, const IluTiles &tiles, const char *stages, const T *f,
                            T *x, const int *done, int *status, unsigned long long timeout_ns);
inline bool is_cpr_type(int pc) {
    return pc == RSV_PC_CPR || pc == RSV_PC_CPR_LEARNED || pc == RSV_PC_CPR_FP || pc == RSV_PC_CPR_FPF ||
           pc == RSV_PC_CPR_FFPF;
}
inline const char *cpr_stages(int pc) {
    return pc == RSV_PC_CPR_FP ? "FP" : pc == RSV_PC_CPR_FPF ? "FPF" : pc == RSV_PC_CPR_FFPF ? "FFPF" : "PF";
}
template <typename T>
cudaError_t cpr_pressure_vcycle(const rsv_mat *A, const Cpr &P, const int *gate);
template <typename T>
cudaError_t cpr_finish(const rsv_mat *A, const Cpr &P, const IluTiles &tiles, const T *f, T *x, const int *done,
                       int *status, unsigned long long timeout_ns);
template <typename T>
cudaError_t cpr_vcycle(const rsv_mat *A, const Cpr &P, const T *b, T *x);

// ---- launchers implemented in ilu_tiles.cu
template <typename T>
cudaError_t tiles_setup(const rsv_mat *A, const double *dinv, IluTiles *T_);
void free_tiles(IluTiles *T_);
template <typename T>
// add0 (optional): z_c[0] += add0[c] on output (carried through the sweeps in the vector's pad slot).
cudaError_t launch_ilu_apply_tiles(const rsv_mat *A, const IluTiles &T_, const T *r, T *z, const int *done,
                                   int *status, unsigned long long timeout_ns, const T *add0 = nullptr);

}  // namespace rsv
