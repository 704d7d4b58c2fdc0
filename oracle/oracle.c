/*
 * CPU FP64 oracle for the reservoir linear-solve path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, sequential
 * definition of what the CUDA library computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the product
 * path never links, calls or falls back to it.  It shares no code, header or
 * constant with the CUDA sources.
 *
 * Every routine follows the paper's definitions (sections cited per routine):
 *   - matrix/vector algebra, Section "Algebraic Operations" (y = aAx + by, <x,y>, ||x||);
 *   - ILU, Section "Restricted Additive Schwarz Method" (LUx = b <=> Ly = b, Ux = y;
 *     ILU(0) is the default local solver in the RAS parameter defaults);
 *   - multigrid, Section "Algebraic Multigrid Methods" (R = P^T, A_{l+1} = R A P,
 *     V-cycle algorithm with pre-smoother, restriction, recursion, prolongation,
 *     post-smoother and exact coarsest solve; defaults 1 cycle, 6 levels, 2 sweeps);
 *   - CPR, Section "CPR-like Preconditioners" (restriction Pi_r, prolongation Pi_p,
 *     CPR-PF algorithm, quasi-IMPES decoupling named in the numerical experiments);
 *   - Krylov solvers, Section "Solvers" (restarted GMRES(m), BiCGSTAB; SOLVER fields
 *     rtol/atol/btol/maxit/restart).
 * Where the paper is silent the readings used are stated beside the code.
 * Parity of every routine is pinned by tests against closed forms, dense
 * linear algebra and invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ESINGULAR 5
#define OR_EBREAKDOWN 6
#define OR_ENOCONV 7
#define OR_ENAN 9

/* Threads of the OpenMP build (the timing baseline); the plain build is
 * sequential and returns 1.  The OpenMP build runs the independent loops
 * (SpMV rows, vector updates, one colour of Gauss-Seidel, stencil products)
 * in parallel; the triangular ILU(0) sweeps stay sequential in natural order.
 * Only its dot products round differently (reduction order). */
int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ BLAS-1 */

/* alpha = <x, y>  (Algebraic Operations) */
double or_dot(int64_t n, const double *x, const double *y) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* alpha = <x, x>^(1/2) */
double or_norm2(int64_t n, const double *x) { return sqrt(or_dot(n, x, x)); }

/* y = alpha x + beta y */
static void axpby(int64_t n, double a, const double *x, double b, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) y[i] = a * x[i] + b * y[i];
}

/* ------------------------------------------------------------- BSR SpMV */

/* y = alpha A x + beta y for a 3x3-block BSR matrix (Algebraic Operations).
 * Blocks are row-major; a row's blocks are summed in ascending column order. */
int or_spmv(int nb, const int32_t *rp, const int32_t *ci, const double *v,
            double alpha, const double *x, double beta, double *y) {
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nb; ++r) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int32_t p = rp[r]; p < rp[r + 1]; ++p) {
            const double *a = v + 9 * (int64_t)p;
            const double *xc = x + 3 * (int64_t)ci[p];
            for (int e = 0; e < 3; ++e)
                for (int f = 0; f < 3; ++f) acc[e] += a[3 * e + f] * xc[f];
        }
        for (int e = 0; e < 3; ++e) {
            double old = (beta == 0.0) ? 0.0 : beta * y[3 * (int64_t)r + e];
            y[3 * (int64_t)r + e] = alpha * acc[e] + old;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------ dense elimination */

/* Solve A X = B (A n x n row-major, B n x nrhs row-major) by Gaussian
 * elimination with partial pivoting.  A and B are overwritten; X lands in B.
 * A pivot with |p| <= 1e-300 reports singularity. */
static int gauss_solve(int n, double *A, double *B, int nrhs) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[(int64_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double t = fabs(A[(int64_t)i * n + k]);
            if (t > best) { best = t; piv = i; }
        }
        if (!(best > 1e-300)) return OR_ESINGULAR;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(int64_t)k * n + j];
                A[(int64_t)k * n + j] = A[(int64_t)piv * n + j];
                A[(int64_t)piv * n + j] = t;
            }
            for (int j = 0; j < nrhs; ++j) {
                double t = B[(int64_t)k * nrhs + j];
                B[(int64_t)k * nrhs + j] = B[(int64_t)piv * nrhs + j];
                B[(int64_t)piv * nrhs + j] = t;
            }
        }
        for (int i = k + 1; i < n; ++i) {
            double l = A[(int64_t)i * n + k] / A[(int64_t)k * n + k];
            if (l == 0.0) continue;
            for (int j = k; j < n; ++j) A[(int64_t)i * n + j] -= l * A[(int64_t)k * n + j];
            for (int j = 0; j < nrhs; ++j) B[(int64_t)i * nrhs + j] -= l * B[(int64_t)k * nrhs + j];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        for (int j = 0; j < nrhs; ++j) {
            double s = B[(int64_t)k * nrhs + j];
            for (int i = k + 1; i < n; ++i) s -= A[(int64_t)k * n + i] * B[(int64_t)i * nrhs + j];
            B[(int64_t)k * nrhs + j] = s / A[(int64_t)k * n + k];
        }
    }
    return OR_OK;
}

/* Dense solve A x = b (A row-major n x n, left untouched). */
int or_dense_solve(int n, const double *A, const double *b, double *x) {
    double *a = (double *)malloc(sizeof(double) * (size_t)n * n);
    if (!a) return OR_ENOMEM;
    memcpy(a, A, sizeof(double) * (size_t)n * n);
    memcpy(x, b, sizeof(double) * (size_t)n);
    int st = gauss_solve(n, a, x, 1);
    free(a);
    return st;
}

/* Inverse of one 3x3 block by elimination against the identity. */
int or_inv3(const double *a, double *ainv) {
    double m[9];
    memcpy(m, a, sizeof m);
    for (int i = 0; i < 9; ++i) ainv[i] = (i % 4 == 0) ? 1.0 : 0.0;
    return gauss_solve(3, m, ainv, 3);
}

static void mat3_vec(const double *a, const double *x, double *y) {
    for (int e = 0; e < 3; ++e) y[e] = a[3 * e] * x[0] + a[3 * e + 1] * x[1] + a[3 * e + 2] * x[2];
}

static void mat3_mul(const double *a, const double *b, double *c) {
    for (int e = 0; e < 3; ++e)
        for (int f = 0; f < 3; ++f)
            c[3 * e + f] = a[3 * e] * b[f] + a[3 * e + 1] * b[3 + f] + a[3 * e + 2] * b[6 + f];
}

static int32_t find_block(const int32_t *rp, const int32_t *ci, int r, int c) {
    for (int32_t p = rp[r]; p < rp[r + 1]; ++p)
        if (ci[p] == c) return p;
    return -1;
}

/* ----------------------------------------------------------- block Jacobi */

/* Setup: dinv_i = (A_ii)^{-1} for every block row. */
int or_bj_setup(int nb, const int32_t *rp, const int32_t *ci, const double *v, double *dinv) {
    for (int r = 0; r < nb; ++r) {
        int32_t p = find_block(rp, ci, r, r);
        if (p < 0) return OR_EINVAL;
        if (or_inv3(v + 9 * (int64_t)p, dinv + 9 * (int64_t)r)) return OR_ESINGULAR;
    }
    return OR_OK;
}

/* Apply: z_i = dinv_i r_i. */
void or_bj_apply(int nb, const double *dinv, const double *r, double *z) {
    for (int i = 0; i < nb; ++i) mat3_vec(dinv + 9 * (int64_t)i, r + 3 * (int64_t)i, z + 3 * (int64_t)i);
}

/* ------------------------------------------------------- block ILU(0) */

/* Block ILU(0) in natural row order, general form over the pattern of A:
 *   for each row i, for each k < i in row i (ascending):
 *       L_ik = A_ik U_kk^{-1};
 *       for each j > k in row k: if (i,j) in pattern(A): A_ij -= L_ik A_kj.
 * The factor overwrites a copy of the values: strict-lower blocks hold L
 * (unit diagonal implied), the rest holds U.  udinv_i = U_ii^{-1}.
 * *offdiag_updates counts updates that hit a block other than the diagonal
 * (zero for the seven-point pattern, whose graph has no triangles). */
int or_bilu0_setup(int nb, const int32_t *rp, const int32_t *ci, const double *v,
                   double *lu, double *udinv, int64_t *offdiag_updates) {
    memcpy(lu, v, sizeof(double) * 9 * (size_t)rp[nb]);
    int64_t off = 0;
    for (int i = 0; i < nb; ++i) {
        for (int32_t pk = rp[i]; pk < rp[i + 1] && ci[pk] < i; ++pk) {
            int k = ci[pk];
            double lik[9];
            mat3_mul(lu + 9 * (int64_t)pk, udinv + 9 * (int64_t)k, lik);
            memcpy(lu + 9 * (int64_t)pk, lik, sizeof lik);
            for (int32_t pj = rp[k]; pj < rp[k + 1]; ++pj) {
                int j = ci[pj];
                if (j <= k) continue;
                int32_t pij = find_block(rp, ci, i, j);
                if (pij < 0) continue;  /* no fill outside the pattern */
                double t[9];
                mat3_mul(lik, lu + 9 * (int64_t)pj, t);
                for (int q = 0; q < 9; ++q) lu[9 * (int64_t)pij + q] -= t[q];
                if (j != i) ++off;
            }
        }
        int32_t pd = find_block(rp, ci, i, i);
        if (pd < 0) return OR_EINVAL;
        if (or_inv3(lu + 9 * (int64_t)pd, udinv + 9 * (int64_t)i)) return OR_ESINGULAR;
    }
    if (offdiag_updates) *offdiag_updates = off;
    return OR_OK;
}

/* Apply z = (LU)^{-1} r: L y = r forward, then U z = y backward. */
void or_bilu0_apply(int nb, const int32_t *rp, const int32_t *ci, const double *lu,
                    const double *udinv, const double *r, double *z) {
    double *y = z; /* y then z in place: row i of the backward sweep only reads rows > i */
    for (int i = 0; i < nb; ++i) {
        double s[3] = {r[3 * (int64_t)i], r[3 * (int64_t)i + 1], r[3 * (int64_t)i + 2]};
        for (int32_t p = rp[i]; p < rp[i + 1] && ci[p] < i; ++p) {
            double t[3];
            mat3_vec(lu + 9 * (int64_t)p, y + 3 * (int64_t)ci[p], t);
            for (int e = 0; e < 3; ++e) s[e] -= t[e];
        }
        for (int e = 0; e < 3; ++e) y[3 * (int64_t)i + e] = s[e];
    }
    for (int i = nb - 1; i >= 0; --i) {
        double s[3] = {y[3 * (int64_t)i], y[3 * (int64_t)i + 1], y[3 * (int64_t)i + 2]};
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (ci[p] <= i) continue;
            double t[3];
            mat3_vec(lu + 9 * (int64_t)p, z + 3 * (int64_t)ci[p], t);
            for (int e = 0; e < 3; ++e) s[e] -= t[e];
        }
        mat3_vec(udinv + 9 * (int64_t)i, s, z + 3 * (int64_t)i);
    }
}

/* ----------------------------------------------- quasi-IMPES and Pi_r / Pi_p */

/* Seven-point scalar stencil storage used for the pressure system:
 * a7[c*7 + s], s = 0:-z 1:-y 2:-x 3:centre 4:+x 5:+y 6:+z (0 where no face). */
static const int SX[7] = {0, 0, -1, 0, 1, 0, 0};
static const int SY[7] = {0, -1, 0, 0, 0, 1, 0};
static const int SZ[7] = {-1, 0, 0, 0, 0, 0, 1};

static int stencil_slot(int di, int dj, int dk) {
    for (int s = 0; s < 7; ++s)
        if (SX[s] == di && SY[s] == dj && SZ[s] == dk) return s;
    return -1;
}

/* Quasi-IMPES weights (diagonal reading of the decoupling named in the
 * experiments): with D = A_ii, w_i = (1, -D01/D11, -D02/D22).  The pressure
 * matrix is the pressure column of the weighted block rows,
 * (A_pp)_ij = sum_r w_i[r] A_ij[r][0], stored as a seven-point stencil. */
/* Decoupling weights and the pressure operator of CPR.  decoupling 0: the
 * quasi-IMPES reading w_c = (1, -D01/D11, -D02/D22); 1: ABF (alternate block
 * factorization, Section "Numerical experiments" names it beside quasi-IMPES),
 * which premultiplies each block row by D^{-1}, so w_c is the first row of
 * D^{-1} = adj(D) / det(D) (D = A_cc); 2: true-IMPES (named beside them), the
 * same with D = C_c, the cell's accumulation block (the time-derivative part
 * of the Jacobian, passed in as acc[nb][3][3]): w_c C_c = (1, 0, 0) removes
 * the secondary unknowns from the accumulation terms.  Every time
 * A_pp(c, l) = w_c . A_cl[:, 0]. */
int or_decouple_setup(int nx, int ny, int nz, const int32_t *rp, const int32_t *ci, const double *v, int decoupling,
                      const double *acc, double *w, double *a7) {
    int nb = nx * ny * nz;
    if (decoupling == 2 && !acc) return OR_EINVAL;
    memset(a7, 0, sizeof(double) * 7 * (size_t)nb);
    for (int c = 0; c < nb; ++c) {
        int32_t pd = find_block(rp, ci, c, c);
        if (pd < 0) return OR_EINVAL;
        /* ABF inverts the diagonal block of A; true-IMPES the cell's accumulation block */
        const double *d = (decoupling == 2) ? acc + 9 * (int64_t)c : v + 9 * (int64_t)pd;
        double *wc = w + 3 * (int64_t)c;
        if (decoupling == 1 || decoupling == 2) {
            /* first row of the adjugate: cofactors of the first column */
            const double c0 = d[4] * d[8] - d[5] * d[7];
            const double c1 = d[5] * d[6] - d[3] * d[8];
            const double c2 = d[3] * d[7] - d[4] * d[6];
            const double det = d[0] * c0 + d[1] * c1 + d[2] * c2;
            if (!(fabs(det) > 1e-300)) return OR_ESINGULAR;
            wc[0] = c0 / det;
            wc[1] = (d[2] * d[7] - d[1] * d[8]) / det;
            wc[2] = (d[1] * d[5] - d[2] * d[4]) / det;
        } else {
            if (!(fabs(d[4]) > 1e-300) || !(fabs(d[8]) > 1e-300)) return OR_ESINGULAR;
            wc[0] = 1.0;
            wc[1] = -d[1] / d[4];
            wc[2] = -d[2] / d[8];
        }
        int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        for (int32_t p = rp[c]; p < rp[c + 1]; ++p) {
            int o = ci[p];
            int oi = o % nx, oj = (o / nx) % ny, ok = o / (nx * ny);
            int s = stencil_slot(oi - i, oj - j, ok - k);
            if (s < 0) return OR_EINVAL;
            const double *a = v + 9 * (int64_t)p;
            a7[7 * (int64_t)c + s] = wc[0] * a[0] + wc[1] * a[3] + wc[2] * a[6];
        }
    }
    return OR_OK;
}

int or_qi_setup(int nx, int ny, int nz, const int32_t *rp, const int32_t *ci, const double *v, double *w, double *a7) {
    return or_decouple_setup(nx, ny, nz, rp, ci, v, 0, NULL, w, a7);
}

/* Pi_r with the decoupling folded in: p_i = w_i . r_i. */
void or_restrict_pressure(int nb, const double *w, const double *r, double *p) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nb; ++i)
        p[i] = w[3 * (int64_t)i] * r[3 * (int64_t)i] + w[3 * (int64_t)i + 1] * r[3 * (int64_t)i + 1] +
               w[3 * (int64_t)i + 2] * r[3 * (int64_t)i + 2];
}

/* Pi_p: x_i = (p_i, 0, 0). */
void or_prolong_pressure(int nb, const double *p, double *x) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nb; ++i) {
        x[3 * (int64_t)i] = p[i];
        x[3 * (int64_t)i + 1] = 0.0;
        x[3 * (int64_t)i + 2] = 0.0;
    }
}

/* y = a7 x  for a seven-point stencil on an nx*ny*nz grid. */
void or_stencil_apply(int nx, int ny, int nz, const double *a7, const double *x, double *y) {
    int nb = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nb; ++c) {
        int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        double s = 0.0;
        for (int q = 0; q < 7; ++q) {
            int ii = i + SX[q], jj = j + SY[q], kk = k + SZ[q];
            if (ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz) continue;
            s += a7[7 * (int64_t)c + q] * x[(int64_t)nx * ny * kk + (int64_t)nx * jj + ii];
        }
        y[c] = s;
    }
}

/* ------------------------------------------------------ geometric multigrid */

/* Galerkin coarse operator A_c = P^T A P for piecewise-constant P on 2x2x2
 * boxes (coarse cell (i/2, j/2, k/2); dims ceil(d/2)).  Entry (I,J) of the
 * product is the sum of fine couplings A_ij with i in box I and j in box J;
 * couplings inside one box add to the coarse centre. */
void or_gmg_coarsen(int nx, int ny, int nz, const double *a7, double *ac7) {
    int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    memset(ac7, 0, sizeof(double) * 7 * (size_t)cx * cy * cz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t c = (int64_t)nx * ny * k + (int64_t)nx * j + i;
                int64_t C = (int64_t)cx * cy * (k / 2) + (int64_t)cx * (j / 2) + i / 2;
                for (int q = 0; q < 7; ++q) {
                    int ii = i + SX[q], jj = j + SY[q], kk = k + SZ[q];
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz) continue;
                    int s = stencil_slot(ii / 2 - i / 2, jj / 2 - j / 2, kk / 2 - k / 2);
                    ac7[7 * C + s] += a7[7 * c + q];
                }
            }
}

/* One Gauss-Seidel sweep over the cells of one colour ((i+j+k) mod 2),
 * visiting them in natural order. */
void or_gs_colour(int nx, int ny, int nz, const double *a7, const double *b, double *x, int colour) {
    /* cells of one colour couple only to the other colour, so the k-planes are independent */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (((i + j + k) & 1) != colour) continue;
                int64_t c = (int64_t)nx * ny * k + (int64_t)nx * j + i;
                double s = b[c];
                for (int q = 0; q < 7; ++q) {
                    if (q == 3) continue;
                    int ii = i + SX[q], jj = j + SY[q], kk = k + SZ[q];
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz) continue;
                    s -= a7[7 * c + q] * x[(int64_t)nx * ny * kk + (int64_t)nx * jj + ii];
                }
                x[c] = s / a7[7 * c + 3];
            }
}

#define OR_MAX_LEVELS 8
typedef struct {
    int nlev;
    int nx[OR_MAX_LEVELS], ny[OR_MAX_LEVELS], nz[OR_MAX_LEVELS];
    double *a7[OR_MAX_LEVELS];
    double *x[OR_MAX_LEVELS], *b[OR_MAX_LEVELS], *r[OR_MAX_LEVELS];
    double *coarse_dense; /* coarsest operator, dense row-major */
    int sweeps;
} or_gmg;

/* Level count rule: halve (ceil) every dimension while the level has more than
 * `max_coarse` cells, up to `max_levels` levels (paper default 6). */
static int gmg_build(or_gmg *g, int nx, int ny, int nz, const double *a7, int max_levels,
                     int max_coarse, int sweeps) {
    memset(g, 0, sizeof *g);
    if (max_levels > OR_MAX_LEVELS) max_levels = OR_MAX_LEVELS;
    g->sweeps = sweeps;
    g->nx[0] = nx; g->ny[0] = ny; g->nz[0] = nz;
    int64_t n0 = (int64_t)nx * ny * nz;
    g->a7[0] = (double *)malloc(sizeof(double) * 7 * n0);
    memcpy(g->a7[0], a7, sizeof(double) * 7 * n0);
    int l = 0;
    while (l + 1 < max_levels && (int64_t)g->nx[l] * g->ny[l] * g->nz[l] > max_coarse) {
        int cx = (g->nx[l] + 1) / 2, cy = (g->ny[l] + 1) / 2, cz = (g->nz[l] + 1) / 2;
        g->nx[l + 1] = cx; g->ny[l + 1] = cy; g->nz[l + 1] = cz;
        g->a7[l + 1] = (double *)malloc(sizeof(double) * 7 * (size_t)cx * cy * cz);
        or_gmg_coarsen(g->nx[l], g->ny[l], g->nz[l], g->a7[l], g->a7[l + 1]);
        ++l;
    }
    g->nlev = l + 1;
    for (int q = 0; q < g->nlev; ++q) {
        size_t n = (size_t)g->nx[q] * g->ny[q] * g->nz[q];
        g->x[q] = (double *)calloc(n, sizeof(double));
        g->b[q] = (double *)calloc(n, sizeof(double));
        g->r[q] = (double *)calloc(n, sizeof(double));
    }
    int L = g->nlev - 1;
    int nc = g->nx[L] * g->ny[L] * g->nz[L];
    g->coarse_dense = (double *)calloc((size_t)nc * nc, sizeof(double));
    for (int c = 0; c < nc; ++c) {
        int i = c % g->nx[L], j = (c / g->nx[L]) % g->ny[L], k = c / (g->nx[L] * g->ny[L]);
        for (int q = 0; q < 7; ++q) {
            int ii = i + SX[q], jj = j + SY[q], kk = k + SZ[q];
            if (ii < 0 || jj < 0 || kk < 0 || ii >= g->nx[L] || jj >= g->ny[L] || kk >= g->nz[L]) continue;
            int o = g->nx[L] * g->ny[L] * kk + g->nx[L] * jj + ii;
            g->coarse_dense[(size_t)c * nc + o] += g->a7[L][7 * (size_t)c + q];
        }
    }
    return OR_OK;
}

static void gmg_free(or_gmg *g) {
    for (int q = 0; q < g->nlev; ++q) { free(g->a7[q]); free(g->x[q]); free(g->b[q]); free(g->r[q]); }
    free(g->coarse_dense);
    memset(g, 0, sizeof *g);
}

/* V-cycle from a zero initial guess on level l (multigrid V-cycle algorithm):
 * pre-smooth (red then black, `sweeps` times), residual, restrict with
 * R = P^T (sum over each 2x2x2 box), recurse, prolong (inject) and add,
 * post-smooth (black then red), exact dense solve on the coarsest level. */
static int gmg_vcycle(or_gmg *g, int l) {
    int nx = g->nx[l], ny = g->ny[l], nz = g->nz[l];
    int64_t n = (int64_t)nx * ny * nz;
    if (l == g->nlev - 1) {
        return or_dense_solve((int)n, g->coarse_dense, g->b[l], g->x[l]);
    }
    memset(g->x[l], 0, sizeof(double) * n);
    for (int s = 0; s < g->sweeps; ++s) {
        or_gs_colour(nx, ny, nz, g->a7[l], g->b[l], g->x[l], 0);
        or_gs_colour(nx, ny, nz, g->a7[l], g->b[l], g->x[l], 1);
    }
    or_stencil_apply(nx, ny, nz, g->a7[l], g->x[l], g->r[l]);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) g->r[l][c] = g->b[l][c] - g->r[l][c];
    int cx = g->nx[l + 1], cy = g->ny[l + 1];
    memset(g->b[l + 1], 0, sizeof(double) * (size_t)cx * cy * g->nz[l + 1]);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                g->b[l + 1][(int64_t)cx * cy * (k / 2) + (int64_t)cx * (j / 2) + i / 2] +=
                    g->r[l][(int64_t)nx * ny * k + (int64_t)nx * j + i];
    int st = gmg_vcycle(g, l + 1);
    if (st) return st;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                g->x[l][(int64_t)nx * ny * k + (int64_t)nx * j + i] +=
                    g->x[l + 1][(int64_t)cx * cy * (k / 2) + (int64_t)cx * (j / 2) + i / 2];
    for (int s = 0; s < g->sweeps; ++s) {
        or_gs_colour(nx, ny, nz, g->a7[l], g->b[l], g->x[l], 1);
        or_gs_colour(nx, ny, nz, g->a7[l], g->b[l], g->x[l], 0);
    }
    return OR_OK;
}

/* Stand-alone V-cycle for tests: e = V(rhs) on the stencil hierarchy. */
int or_gmg_vcycle(int nx, int ny, int nz, const double *a7, int max_levels, int max_coarse,
                  int sweeps, const double *rhs, double *e, int *nlev_out) {
    or_gmg g;
    gmg_build(&g, nx, ny, nz, a7, max_levels, max_coarse, sweeps);
    memcpy(g.b[0], rhs, sizeof(double) * (size_t)nx * ny * nz);
    int st = gmg_vcycle(&g, 0);
    memcpy(e, g.x[0], sizeof(double) * (size_t)nx * ny * nz);
    if (nlev_out) *nlev_out = g.nlev;
    gmg_free(&g);
    return st;
}


/* ---------------------------------------------------- algebraic multigrid */

/* Algebraic coarsening for the pressure stage (Section "Algebraic Multigrid
 * Methods", AMG setup algorithm: strength matrix, coarse set as a subset of
 * the fine points, prolongation, R = P^T, Galerkin product, smoothers; and
 * the same V-cycle algorithm as the geometric hierarchy).  The readings:
 *   - strength: j != i strongly influences i when -a_ij >= theta max_{k != i}
 *     (-a_ik), theta = 0.5 (the strength threshold of the default-parameter
 *     figure); no strong connections when that maximum is <= 0;
 *   - coarse set: PMIS (one of the parallel coarsenings the section names).
 *     Measure lambda_i = |{k : i in S_k}| + u_i with u_i a counter-based
 *     uniform in [0, 1) (splitmix64 of the point index).  Points that no
 *     point depends on (lambda_i < 1) start as F.  Then, in rounds from the
 *     previous round's state: an undecided point whose measure exceeds every
 *     undecided strong neighbour's (S_i and S_i^T) becomes C; afterwards each
 *     undecided point that strongly depends on a C point becomes F;
 *   - prolongation: identity on C points; direct interpolation on F points,
 *     w_ij = -alpha_i a_ij / a_ii for j in C_i = S_i n C, with
 *     alpha_i = sum_{k != i} a_ik / sum_{k in C_i} a_ik (a zero row when C_i
 *     is empty or that sum vanishes);
 *   - smoother: l1-Jacobi, x += D^{-1} (b - A x) with D_ii = sum_j |a_ij|,
 *     `sweeps` times before and after the coarse correction (the hybrid
 *     Gauss-Seidel of the defaults is Jacobi between blocks; with one row per
 *     block it is Jacobi, and the l1 diagonal keeps it convergent without a
 *     damping parameter);
 *   - levels: coarsen while a level has more than max_coarse points, up to
 *     max_levels levels, and stop when a round keeps more than 90% of the
 *     points; the coarsest level is solved exactly (dense LU). */
typedef struct { int n; int *rp, *ci; double *v; } or_csr;

static void csr_free(or_csr *a) { free(a->rp); free(a->ci); free(a->v); memset(a, 0, sizeof *a); }

static double amg_uniform(int64_t i) {
    uint64_t z = (uint64_t)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* Strength pattern: s_rp/s_ci list, per row, the columns j in S_i (ascending). */
static void amg_strength(const or_csr *A, double theta, int **s_rp, int **s_ci) {
    int n = A->n;
    int *rp = (int *)calloc((size_t)n + 1, sizeof(int));
    int *ci = (int *)malloc(sizeof(int) * (size_t)(A->rp[n] > 0 ? A->rp[n] : 1));
    for (int i = 0; i < n; ++i) {
        double mx = 0.0;
        for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
            if (A->ci[p] != i && -A->v[p] > mx) mx = -A->v[p];
        rp[i + 1] = rp[i];
        if (!(mx > 0.0)) continue;
        for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
            if (A->ci[p] != i && -A->v[p] >= theta * mx) ci[rp[i + 1]++] = A->ci[p];
    }
    *s_rp = rp;
    *s_ci = ci;
}

/* PMIS: cf[i] = 1 (C) or -1 (F). */
static void amg_pmis(int n, const int *s_rp, const int *s_ci, int *cf) {
    int *cnt = (int *)calloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; ++i)
        for (int p = s_rp[i]; p < s_rp[i + 1]; ++p) cnt[s_ci[p]]++;
    /* transpose of S: t_ci lists the points k with i in S_k */
    int *t_rp = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int i = 0; i < n; ++i) t_rp[i + 1] = t_rp[i] + cnt[i];
    int *t_ci = (int *)malloc(sizeof(int) * (size_t)(t_rp[n] > 0 ? t_rp[n] : 1));
    int *fill = (int *)calloc((size_t)n, sizeof(int));
    for (int k = 0; k < n; ++k)
        for (int p = s_rp[k]; p < s_rp[k + 1]; ++p) {
            int i = s_ci[p];
            t_ci[t_rp[i] + fill[i]++] = k;
        }
    double *lam = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        lam[i] = cnt[i] + amg_uniform(i);
        cf[i] = lam[i] < 1.0 ? -1 : 0;
    }
    int *newc = (int *)calloc((size_t)n, sizeof(int));
    for (;;) {
        int undecided = 0;
        for (int i = 0; i < n; ++i) undecided += cf[i] == 0;
        if (!undecided) break;
        for (int i = 0; i < n; ++i) {
            newc[i] = 0;
            if (cf[i] != 0) continue;
            int best = 1;
            for (int p = s_rp[i]; p < s_rp[i + 1] && best; ++p)
                if (cf[s_ci[p]] == 0 && lam[s_ci[p]] >= lam[i]) best = 0;
            for (int p = t_rp[i]; p < t_rp[i + 1] && best; ++p)
                if (cf[t_ci[p]] == 0 && lam[t_ci[p]] >= lam[i]) best = 0;
            newc[i] = best;
        }
        for (int i = 0; i < n; ++i)
            if (newc[i]) cf[i] = 1;
        for (int i = 0; i < n; ++i) {
            if (cf[i] != 0) continue;
            for (int p = s_rp[i]; p < s_rp[i + 1]; ++p)
                if (cf[s_ci[p]] == 1) { cf[i] = -1; break; }
        }
    }
    free(cnt); free(t_rp); free(t_ci); free(fill); free(lam); free(newc);
}

/* Direct interpolation P (n x nc, CSR, columns ascending); cidx[i] = coarse index of C point i. */
static void amg_interp(const or_csr *A, const int *s_rp, const int *s_ci, const int *cf, const int *cidx,
                       or_csr *P) {
    int n = A->n;
    P->n = n;
    P->rp = (int *)calloc((size_t)n + 1, sizeof(int));
    P->ci = (int *)malloc(sizeof(int) * (size_t)(s_rp[n] + n + 1));
    P->v = (double *)malloc(sizeof(double) * (size_t)(s_rp[n] + n + 1));
    int q = 0;
    for (int i = 0; i < n; ++i) {
        if (cf[i] == 1) {
            P->ci[q] = cidx[i];
            P->v[q++] = 1.0;
        } else {
            double aii = 0.0, sum_n = 0.0, sum_c = 0.0;
            for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
                if (A->ci[p] == i) { aii = A->v[p]; continue; }
                sum_n += A->v[p];
            }
            /* strong C neighbours, with their coefficients a_ij */
            for (int p = s_rp[i]; p < s_rp[i + 1]; ++p) {
                int j = s_ci[p];
                if (cf[j] != 1) continue;
                for (int r = A->rp[i]; r < A->rp[i + 1]; ++r)
                    if (A->ci[r] == j) sum_c += A->v[r];
            }
            if (sum_c != 0.0 && aii != 0.0) {
                double alpha = sum_n / sum_c;
                for (int p = s_rp[i]; p < s_rp[i + 1]; ++p) {
                    int j = s_ci[p];
                    if (cf[j] != 1) continue;
                    for (int r = A->rp[i]; r < A->rp[i + 1]; ++r)
                        if (A->ci[r] == j) {
                            P->ci[q] = cidx[j];
                            P->v[q++] = -alpha * A->v[r] / aii;
                        }
                }
            }
        }
        P->rp[i + 1] = q;
    }
}

/* Galerkin product Ac = P^T A P (nc x nc, CSR, columns ascending).  Entry
 * (I, J) sums P_fI a_fk P_kJ over fine rows f (ascending), their entries k
 * (row order) and P's entries in row k (row order). */
static void amg_rap(const or_csr *A, const or_csr *P, int nc, or_csr *Ac) {
    int n = A->n;
    double *acc = (double *)calloc((size_t)nc, sizeof(double));
    int *mark = (int *)malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    for (int J = 0; J < nc; ++J) mark[J] = -1;
    /* P^T as lists of (f, P_fI) per coarse row I, f ascending */
    int *t_rp = (int *)calloc((size_t)nc + 1, sizeof(int));
    for (int f = 0; f < n; ++f)
        for (int p = P->rp[f]; p < P->rp[f + 1]; ++p) t_rp[P->ci[p] + 1]++;
    for (int I = 0; I < nc; ++I) t_rp[I + 1] += t_rp[I];
    int *t_f = (int *)malloc(sizeof(int) * (size_t)(t_rp[nc] > 0 ? t_rp[nc] : 1));
    double *t_v = (double *)malloc(sizeof(double) * (size_t)(t_rp[nc] > 0 ? t_rp[nc] : 1));
    int *fill = (int *)calloc((size_t)nc, sizeof(int));
    for (int f = 0; f < n; ++f)
        for (int p = P->rp[f]; p < P->rp[f + 1]; ++p) {
            int I = P->ci[p];
            t_f[t_rp[I] + fill[I]] = f;
            t_v[t_rp[I] + fill[I]++] = P->v[p];
        }
    int cap = 16 * (nc > 0 ? nc : 1);
    Ac->n = nc;
    Ac->rp = (int *)calloc((size_t)nc + 1, sizeof(int));
    Ac->ci = (int *)malloc(sizeof(int) * (size_t)cap);
    Ac->v = (double *)malloc(sizeof(double) * (size_t)cap);
    int *cols = (int *)malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    int q = 0;
    for (int I = 0; I < nc; ++I) {
        int nnz = 0;
        for (int t = t_rp[I]; t < t_rp[I + 1]; ++t) {
            int f = t_f[t];
            double pf = t_v[t];
            for (int a = A->rp[f]; a < A->rp[f + 1]; ++a) {
                int k = A->ci[a];
                for (int b = P->rp[k]; b < P->rp[k + 1]; ++b) {
                    int J = P->ci[b];
                    if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; cols[nnz++] = J; }
                    acc[J] += pf * A->v[a] * P->v[b];
                }
            }
        }
        /* ascending columns */
        for (int x = 1; x < nnz; ++x) {
            int c = cols[x], y = x - 1;
            while (y >= 0 && cols[y] > c) { cols[y + 1] = cols[y]; --y; }
            cols[y + 1] = c;
        }
        if (q + nnz > cap) {
            while (q + nnz > cap) cap *= 2;
            Ac->ci = (int *)realloc(Ac->ci, sizeof(int) * (size_t)cap);
            Ac->v = (double *)realloc(Ac->v, sizeof(double) * (size_t)cap);
        }
        for (int x = 0; x < nnz; ++x) {
            Ac->ci[q] = cols[x];
            Ac->v[q++] = acc[cols[x]];
        }
        Ac->rp[I + 1] = q;
    }
    free(acc); free(mark); free(t_rp); free(t_f); free(t_v); free(fill); free(cols);
}

#define OR_AMG_MAX 8
typedef struct {
    int nlev, sweeps;
    or_csr A[OR_AMG_MAX], P[OR_AMG_MAX];  /* P[l]: level l -> l+1 */
    int *cf[OR_AMG_MAX];                  /* C/F splitting of level l (1 C, -1 F) */
    double *dl1[OR_AMG_MAX];              /* l1 row norms */
    double *x[OR_AMG_MAX], *b[OR_AMG_MAX], *r[OR_AMG_MAX];
    double *coarse_dense;
} or_amg;

static void amg_free(or_amg *g) {
    for (int l = 0; l < g->nlev; ++l) {
        csr_free(&g->A[l]);
        csr_free(&g->P[l]);
        free(g->cf[l]);
        free(g->dl1[l]); free(g->x[l]); free(g->b[l]); free(g->r[l]);
    }
    free(g->coarse_dense);
    memset(g, 0, sizeof *g);
}

/* Build the hierarchy from the seven-point pressure stencil a7 (slots -z,-y,-x,centre,+x,+y,+z). */
static int amg_build(or_amg *g, int nx, int ny, int nz, const double *a7, int max_levels, int max_coarse,
                     int sweeps) {
    memset(g, 0, sizeof *g);
    if (max_levels > OR_AMG_MAX) max_levels = OR_AMG_MAX;
    g->sweeps = sweeps;
    int n0 = nx * ny * nz;
    or_csr *A = &g->A[0];
    A->n = n0;
    A->rp = (int *)calloc((size_t)n0 + 1, sizeof(int));
    A->ci = (int *)malloc(sizeof(int) * 7 * (size_t)n0);
    A->v = (double *)malloc(sizeof(double) * 7 * (size_t)n0);
    int q = 0;
    for (int c = 0; c < n0; ++c) {
        int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        for (int s = 0; s < 7; ++s) {  /* slot order is ascending column order */
            int ii = i + SX[s], jj = j + SY[s], kk = k + SZ[s];
            if (ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz) continue;
            A->ci[q] = nx * ny * kk + nx * jj + ii;
            A->v[q++] = a7[7 * (size_t)c + s];
        }
        A->rp[c + 1] = q;
    }
    int l = 0;
    while (l + 1 < max_levels && g->A[l].n > max_coarse) {
        int *s_rp, *s_ci;
        amg_strength(&g->A[l], 0.5, &s_rp, &s_ci);
        int n = g->A[l].n;
        int *cf = (int *)malloc(sizeof(int) * (size_t)n), *cidx = (int *)malloc(sizeof(int) * (size_t)n);
        amg_pmis(n, s_rp, s_ci, cf);
        int nc = 0;
        for (int i = 0; i < n; ++i) cidx[i] = cf[i] == 1 ? nc++ : -1;
        if (nc == 0 || nc > 0.9 * n) { free(s_rp); free(s_ci); free(cf); free(cidx); break; }
        amg_interp(&g->A[l], s_rp, s_ci, cf, cidx, &g->P[l]);
        amg_rap(&g->A[l], &g->P[l], nc, &g->A[l + 1]);
        g->cf[l] = cf;
        free(s_rp); free(s_ci); free(cidx);
        ++l;
    }
    g->nlev = l + 1;
    for (int q2 = 0; q2 < g->nlev; ++q2) {
        int n = g->A[q2].n;
        g->dl1[q2] = (double *)calloc((size_t)n, sizeof(double));
        for (int i = 0; i < n; ++i)
            for (int p = g->A[q2].rp[i]; p < g->A[q2].rp[i + 1]; ++p) g->dl1[q2][i] += fabs(g->A[q2].v[p]);
        g->x[q2] = (double *)calloc((size_t)n, sizeof(double));
        g->b[q2] = (double *)calloc((size_t)n, sizeof(double));
        g->r[q2] = (double *)calloc((size_t)n, sizeof(double));
    }
    int L = g->nlev - 1, nc = g->A[L].n;
    if (nc > 4096) return OR_EINVAL;
    g->coarse_dense = (double *)calloc((size_t)nc * nc, sizeof(double));
    for (int i = 0; i < nc; ++i)
        for (int p = g->A[L].rp[i]; p < g->A[L].rp[i + 1]; ++p) g->coarse_dense[(size_t)i * nc + g->A[L].ci[p]] += g->A[L].v[p];
    return OR_OK;
}

static void csr_residual(const or_csr *A, const double *b, const double *x, double *r) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; ++i) {
        double s = 0.0;
        for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * x[A->ci[p]];
        r[i] = b[i] - s;
    }
}

static int amg_vcycle(or_amg *g, int l) {
    const or_csr *A = &g->A[l];
    int n = A->n;
    if (l == g->nlev - 1) return or_dense_solve(n, g->coarse_dense, g->b[l], g->x[l]);
    memset(g->x[l], 0, sizeof(double) * (size_t)n);
    for (int s = 0; s < g->sweeps; ++s) {
        csr_residual(A, g->b[l], g->x[l], g->r[l]);
        for (int i = 0; i < n; ++i) g->x[l][i] += g->r[l][i] / g->dl1[l][i];
    }
    csr_residual(A, g->b[l], g->x[l], g->r[l]);
    const or_csr *P = &g->P[l];
    int nc = g->A[l + 1].n;
    memset(g->b[l + 1], 0, sizeof(double) * (size_t)nc);
    for (int f = 0; f < n; ++f)  /* b_{l+1} = P^T r */
        for (int p = P->rp[f]; p < P->rp[f + 1]; ++p) g->b[l + 1][P->ci[p]] += P->v[p] * g->r[l][f];
    int st = amg_vcycle(g, l + 1);
    if (st) return st;
    for (int f = 0; f < n; ++f) {  /* x += P x_{l+1} */
        double s = 0.0;
        for (int p = P->rp[f]; p < P->rp[f + 1]; ++p) s += P->v[p] * g->x[l + 1][P->ci[p]];
        g->x[l][f] += s;
    }
    for (int s = 0; s < g->sweeps; ++s) {
        csr_residual(A, g->b[l], g->x[l], g->r[l]);
        for (int i = 0; i < n; ++i) g->x[l][i] += g->r[l][i] / g->dl1[l][i];
    }
    return OR_OK;
}

/* Stand-alone AMG pieces for tests.  or_amg_hierarchy: level count, and per
 * level its size and nonzeros (int[2 * OR_AMG_MAX]).  or_amg_vcycle: one
 * V-cycle e = V(rhs) from a zero guess. */
int or_amg_hierarchy(int nx, int ny, int nz, const double *a7, int max_levels, int max_coarse, int *sizes) {
    or_amg g;
    int st = amg_build(&g, nx, ny, nz, a7, max_levels, max_coarse, 2);
    int nl = g.nlev;
    for (int l = 0; l < nl; ++l) { sizes[2 * l] = g.A[l].n; sizes[2 * l + 1] = g.A[l].rp[g.A[l].n]; }
    amg_free(&g);
    return st ? -st : nl;
}

int or_amg_vcycle(int nx, int ny, int nz, const double *a7, int max_levels, int max_coarse, int sweeps,
                  const double *rhs, double *e, int *nlev_out) {
    or_amg g;
    int st = amg_build(&g, nx, ny, nz, a7, max_levels, max_coarse, sweeps);
    if (!st) {
        memcpy(g.b[0], rhs, sizeof(double) * (size_t)nx * ny * nz);
        st = amg_vcycle(&g, 0);
        memcpy(e, g.x[0], sizeof(double) * (size_t)nx * ny * nz);
    }
    if (nlev_out) *nlev_out = g.nlev;
    amg_free(&g);
    return st;
}

/* Level l's strength pattern, C/F splitting, prolongation and coarse operator
 * for tests: copies into caller arrays sized by or_amg_hierarchy's counts.
 * cf[n_l]; P as (rp[n_l+1], ci, v) with at most nnzP entries (returned);
 * Ac as (rp[nc+1], ci, v). */
int or_amg_level(int nx, int ny, int nz, const double *a7, int max_levels, int max_coarse, int level, int *cf,
                 int *p_rp, int *p_ci, double *p_v, int *a_rp, int *a_ci, double *a_v) {
    or_amg g;
    int st = amg_build(&g, nx, ny, nz, a7, max_levels, max_coarse, 2);
    int nnzp = -1;
    if (!st && level + 1 < g.nlev) {
        const or_csr *P = &g.P[level], *Ac = &g.A[level + 1];
        int n = g.A[level].n;
        for (int i = 0; i < n; ++i) {
            cf[i] = g.cf[level][i];
            p_rp[i] = P->rp[i];
        }
        p_rp[n] = P->rp[n];
        for (int p = 0; p < P->rp[n]; ++p) { p_ci[p] = P->ci[p]; p_v[p] = P->v[p]; }
        for (int I = 0; I <= Ac->n; ++I) a_rp[I] = Ac->rp[I];
        for (int p = 0; p < Ac->rp[Ac->n]; ++p) { a_ci[p] = Ac->ci[p]; a_v[p] = Ac->v[p]; }
        nnzp = P->rp[n];
    }
    amg_free(&g);
    return st ? -st : nnzp;
}

/* ------------------------------------------------------------ system + PCs */

enum { PC_NONE = 0, PC_BJACOBI = 1, PC_BILU0 = 2, PC_CPR = 3, PC_CPR_FP = 5, PC_CPR_FPF = 6, PC_CPR_FFPF = 7 };
static int is_cpr(int pc) { return pc == PC_CPR || pc == PC_CPR_FP || pc == PC_CPR_FPF || pc == PC_CPR_FFPF; }

typedef struct {
    int nx, ny, nz, nb;
    const int32_t *rp, *ci;
    double *v;        /* owned copy of the values (float-rounded when requested) */
    int pc;
    double *dinv;     /* block Jacobi */
    double *lu, *udinv; /* block ILU(0) */
    double *w, *a7;   /* decoupling weights, pressure stencil */
    double *acc;      /* accumulation blocks [nb][3][3] (true-IMPES), or NULL */
    int coarsening;   /* pressure hierarchy: 0 geometric (GMG), 1 algebraic (AMG) */
    or_amg amg;
    or_gmg gmg;
    double *tmp_p, *tmp_x, *tmp_r;
    int64_t pc_applies;
} or_system;

static double round_f32(double x) { return (double)(float)x; }

/* Create a system; float_round != 0 rounds every matrix value to float
 * (the FP32 copy used by the inner solves of iterative refinement). */
or_system *or_create(int nx, int ny, int nz, const int32_t *rp, const int32_t *ci, const double *v,
                     int float_round) {
    or_system *s = (or_system *)calloc(1, sizeof(or_system));
    if (!s) return NULL;
    s->nx = nx; s->ny = ny; s->nz = nz; s->nb = nx * ny * nz;
    s->rp = rp; s->ci = ci;
    size_t nv = 9 * (size_t)rp[s->nb];
    s->v = (double *)malloc(sizeof(double) * nv);
    for (size_t q = 0; q < nv; ++q) s->v[q] = float_round ? round_f32(v[q]) : v[q];
    return s;
}

void or_destroy(or_system *s) {
    if (!s) return;
    free(s->v); free(s->dinv); free(s->lu); free(s->udinv); free(s->w); free(s->a7); free(s->acc);
    free(s->tmp_p); free(s->tmp_x); free(s->tmp_r);
    if (s->gmg.nlev) gmg_free(&s->gmg);
    if (s->amg.nlev) amg_free(&s->amg);
    free(s);
}

/* Preconditioner setup.  pc: 0 none, 1 block Jacobi, 2 block ILU(0),
 * 3 CPR-PF (quasi-IMPES + GMG V-cycle pressure stage, then block ILU(0)),
 * 5 CPR-FP, 6 CPR-FPF, 7 CPR-FFPF (the same two stages in the other orders).
 * float_round != 0 rounds the stored factors to float after setup; decoupling:
 * 0 quasi-IMPES, 1 ABF (CPR only). */
/* Accumulation blocks for true-IMPES decoupling (nb blocks of 3x3, copied). */
void or_set_accumulation(or_system *s, const double *acc) {
    free(s->acc);
    s->acc = NULL;
    if (!acc) return;
    s->acc = (double *)malloc(sizeof(double) * 9 * (size_t)s->nb);
    memcpy(s->acc, acc, sizeof(double) * 9 * (size_t)s->nb);
}

int or_setup(or_system *s, int pc, int gmg_levels, int gmg_coarse, int gmg_sweeps, int float_round, int decoupling) {
    int nb = s->nb;
    s->pc = pc;
    int st = OR_OK;
    if (pc == PC_BJACOBI) {
        s->dinv = (double *)malloc(sizeof(double) * 9 * (size_t)nb);
        st = or_bj_setup(nb, s->rp, s->ci, s->v, s->dinv);
        if (float_round)
            for (size_t q = 0; q < 9 * (size_t)nb; ++q) s->dinv[q] = round_f32(s->dinv[q]);
    }
    if (pc == PC_BILU0 || is_cpr(pc)) {
        s->lu = (double *)malloc(sizeof(double) * 9 * (size_t)s->rp[nb]);
        s->udinv = (double *)malloc(sizeof(double) * 9 * (size_t)nb);
        int64_t off = 0;
        st = or_bilu0_setup(nb, s->rp, s->ci, s->v, s->lu, s->udinv, &off);
        if (float_round) {
            for (size_t q = 0; q < 9 * (size_t)s->rp[nb]; ++q) s->lu[q] = round_f32(s->lu[q]);
            for (size_t q = 0; q < 9 * (size_t)nb; ++q) s->udinv[q] = round_f32(s->udinv[q]);
        }
    }
    if (st) return st;
    if (is_cpr(pc)) {
        s->w = (double *)malloc(sizeof(double) * 3 * (size_t)nb);
        s->a7 = (double *)malloc(sizeof(double) * 7 * (size_t)nb);
        st = or_decouple_setup(s->nx, s->ny, s->nz, s->rp, s->ci, s->v, decoupling, s->acc, s->w, s->a7);
        if (st) return st;
        if (float_round) {
            for (size_t q = 0; q < 3 * (size_t)nb; ++q) s->w[q] = round_f32(s->w[q]);
            for (size_t q = 0; q < 7 * (size_t)nb; ++q) s->a7[q] = round_f32(s->a7[q]);
        }
        if (s->coarsening == 1) {
            st = amg_build(&s->amg, s->nx, s->ny, s->nz, s->a7, gmg_levels, gmg_coarse, gmg_sweeps);
            if (st) return st;
            if (float_round)
                for (int l = 0; l < s->amg.nlev; ++l) {
                    or_csr *A = &s->amg.A[l], *P = &s->amg.P[l];
                    for (int p = 0; p < A->rp[A->n]; ++p) A->v[p] = round_f32(A->v[p]);
                    if (P->rp)
                        for (int p = 0; p < P->rp[P->n]; ++p) P->v[p] = round_f32(P->v[p]);
                    for (int i = 0; i < A->n; ++i) s->amg.dl1[l][i] = round_f32(s->amg.dl1[l][i]);
                }
        } else {
            gmg_build(&s->gmg, s->nx, s->ny, s->nz, s->a7, gmg_levels, gmg_coarse, gmg_sweeps);
        }
        if (float_round && s->coarsening != 1)
            for (int l = 1; l < s->gmg.nlev; ++l)
                for (size_t q = 0; q < 7 * (size_t)s->gmg.nx[l] * s->gmg.ny[l] * s->gmg.nz[l]; ++q)
                    s->gmg.a7[l][q] = round_f32(s->gmg.a7[l][q]);
        s->tmp_p = (double *)malloc(sizeof(double) * (size_t)nb);
        s->tmp_x = (double *)malloc(sizeof(double) * 3 * (size_t)nb);
        s->tmp_r = (double *)malloc(sizeof(double) * 3 * (size_t)nb);
    }
    return st;
}

/* CPR-PF in its two-stage multiplicative form (the printed listing overwrites
 * x and reuses f; the reading here is the standard one):
 *   x = Pi_p M_g^{-1} Pi_r f;  r = f - A x;  x = x + ILU0^{-1} r. */
/* The pressure stage's solve on its right-hand side / solution buffers. */
static double *pstage_b(or_system *s) { return s->coarsening == 1 ? s->amg.b[0] : s->gmg.b[0]; }
static double *pstage_x(or_system *s) { return s->coarsening == 1 ? s->amg.x[0] : s->gmg.x[0]; }
static int pstage_vcycle(or_system *s) { return s->coarsening == 1 ? amg_vcycle(&s->amg, 0) : gmg_vcycle(&s->gmg, 0); }

void or_set_coarsening(or_system *s, int mode) { s->coarsening = mode; }

static int cpr_apply(or_system *s, const double *f, double *x) {
    int nb = s->nb;
    or_restrict_pressure(nb, s->w, f, pstage_b(s));
    int st = pstage_vcycle(s);
    if (st) return st;
    or_prolong_pressure(nb, pstage_x(s), x);
    memcpy(s->tmp_r, f, sizeof(double) * 3 * (size_t)nb);
    or_spmv(nb, s->rp, s->ci, s->v, -1.0, x, 1.0, s->tmp_r);
    or_bilu0_apply(nb, s->rp, s->ci, s->lu, s->udinv, s->tmp_r, s->tmp_x);
    for (int64_t q = 0; q < 3 * (int64_t)nb; ++q) x[q] += s->tmp_x[q];
    return OR_OK;
}

/* The CPR orders of Section "CPR-like preconditioners" (Algorithms CPR-FP,
 * CPR-FPF, CPR-FFPF).  Notation: R(A)^{-1} is the full stage (RAS on one
 * subdomain: block ILU(0) of A), M_g(A_pp)^{-1} the pressure solve (one GMG
 * V-cycle), Pi_r / Pi_p the pressure restriction and prolongation.  Each
 * algorithm starts with x = (first stage) f and then, for every later stage,
 * forms r = f - A x and adds that stage applied to r:
 *   FP:   x = R^{-1} f;  r = f - Ax;  x += Pi_p M_g^{-1} Pi_r r
 *   FPF:  FP, then r = f - Ax;  x += R^{-1} r
 *   FFPF: x = R^{-1} f;  r = f - Ax;  x += R^{-1} r;  r = f - Ax;
 *         x += Pi_p M_g^{-1} Pi_r r;  r = f - Ax;  x += R^{-1} r
 * `stages` spells the order, one letter per stage ('F' full, 'P' pressure). */
static void stage_full(or_system *s, const double *r, double *y) {
    or_bilu0_apply(s->nb, s->rp, s->ci, s->lu, s->udinv, r, y);
}
static int stage_pressure(or_system *s, const double *r, double *y) {
    or_restrict_pressure(s->nb, s->w, r, pstage_b(s));
    int st = pstage_vcycle(s);
    if (st) return st;
    or_prolong_pressure(s->nb, pstage_x(s), y);
    return OR_OK;
}
static int cpr_apply_order(or_system *s, const char *stages, const double *f, double *x) {
    int64_t n = 3 * (int64_t)s->nb;
    double *r = s->tmp_r, *y = s->tmp_x;
    for (int q = 0; stages[q]; ++q) {
        const double *src = f;
        if (q > 0) { /* r = f - A x */
            memcpy(r, f, sizeof(double) * (size_t)n);
            or_spmv(s->nb, s->rp, s->ci, s->v, -1.0, x, 1.0, r);
            src = r;
        }
        if (stages[q] == 'F') {
            stage_full(s, src, y);
        } else {
            int st = stage_pressure(s, src, y);
            if (st) return st;
        }
        for (int64_t i = 0; i < n; ++i) x[i] = (q == 0 ? 0.0 : x[i]) + y[i];
    }
    return OR_OK;
}

/* z = M^{-1} r for the configured preconditioner. */
int or_pc_apply(or_system *s, const double *r, double *z) {
    int64_t n = 3 * (int64_t)s->nb;
    s->pc_applies++;
    switch (s->pc) {
    case PC_NONE: memcpy(z, r, sizeof(double) * n); return OR_OK;
    case PC_BJACOBI: or_bj_apply(s->nb, s->dinv, r, z); return OR_OK;
    case PC_BILU0: or_bilu0_apply(s->nb, s->rp, s->ci, s->lu, s->udinv, r, z); return OR_OK;
    case PC_CPR: return cpr_apply(s, r, z);
    case PC_CPR_FP: return cpr_apply_order(s, "FP", r, z);
    case PC_CPR_FPF: return cpr_apply_order(s, "FPF", r, z);
    case PC_CPR_FFPF: return cpr_apply_order(s, "FFPF", r, z);
    }
    return OR_EINVAL;
}

void or_get_factors(const or_system *s, double *udinv, double *w, double *a7) {
    if (udinv && s->udinv) memcpy(udinv, s->udinv, sizeof(double) * 9 * (size_t)s->nb);
    if (udinv && s->dinv) memcpy(udinv, s->dinv, sizeof(double) * 9 * (size_t)s->nb);
    if (w && s->w) memcpy(w, s->w, sizeof(double) * 3 * (size_t)s->nb);
    if (a7 && s->a7) memcpy(a7, s->a7, sizeof(double) * 7 * (size_t)s->nb);
}

int or_gmg_levels(const or_system *s) { return s->coarsening == 1 ? s->amg.nlev : s->gmg.nlev; }

/* ------------------------------------------------------------------ GMRES */

/* Restarted, right-preconditioned GMRES(m) (Saad's form) with modified
 * Gram-Schmidt Arnoldi and Givens rotations; flexible != 0 keeps
 * z_j = M^{-1} v_j (FGMRES) and updates x += Z y, otherwise x += M^{-1}(V y).
 * Convergence: |g_{j+1}| <= rtol ||b|| ends a cycle; the true residual
 * ||b - A x|| is then recomputed and a new cycle starts unless it also meets
 * the tolerance.  iters counts Arnoldi steps over all cycles.
 * stats[0] = iterations, stats[1] = restarts (cycles), stats[2] = final true
 * relative residual, stats[3] = preconditioner applications. */
int or_gmres(or_system *s, const double *b, double *x, int m, double rtol, int maxit, int flexible,
             double *stats) {
    int64_t n = 3 * (int64_t)s->nb;
    double *V = (double *)malloc(sizeof(double) * (size_t)(m + 1) * n);
    double *Z = flexible ? (double *)malloc(sizeof(double) * (size_t)m * n) : NULL;
    double *w = (double *)malloc(sizeof(double) * n);
    double *t = (double *)malloc(sizeof(double) * n);
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double *)calloc(m, sizeof(double)), *sn = (double *)calloc(m, sizeof(double));
    double *g = (double *)calloc(m + 1, sizeof(double)), *y = (double *)calloc(m, sizeof(double));
    double bnorm = or_norm2(n, b);
    double tol = rtol * bnorm;
    int iters = 0, cycles = 0, st = OR_ENOCONV;
    s->pc_applies = 0;
    for (;;) {
        memcpy(w, b, sizeof(double) * n);
        or_spmv(s->nb, s->rp, s->ci, s->v, -1.0, x, 1.0, w);
        double beta = or_norm2(n, w);
        if (!isfinite(beta)) { st = OR_ENAN; break; }
        if (beta <= tol) { st = OR_OK; break; }
        if (iters >= maxit) { st = OR_ENOCONV; break; }
        ++cycles;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; ++q) V[q] = w[q] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            double *vj = V + (size_t)j * n;
            double *zj = flexible ? Z + (size_t)j * n : t;
            int ps = or_pc_apply(s, vj, zj);
            if (ps) { st = ps; goto done; }
            or_spmv(s->nb, s->rp, s->ci, s->v, 1.0, zj, 0.0, w);
            ++iters;
            for (int i = 0; i <= j; ++i) {
                double h = or_dot(n, w, V + (size_t)i * n);
                H[(size_t)i * m + j] = h;
                axpby(n, -h, V + (size_t)i * n, 1.0, w);
            }
            double hn = or_norm2(n, w);
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
            double rho = hypot(a, bb);
            if (!(rho > 0.0) || !isfinite(rho)) { st = isfinite(rho) ? OR_EBREAKDOWN : OR_ENAN; goto done; }
            cs[j] = a / rho;
            sn[j] = bb / rho;
            H[(size_t)j * m + j] = rho;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jend = j + 1;
            int lucky = !(hn > 0.0);
            if (!lucky) {
#pragma omp parallel for schedule(static)
                for (int64_t q = 0; q < n; ++q) V[(size_t)(j + 1) * n + q] = w[q] / hn;
            }
            if (fabs(g[j + 1]) <= tol || iters >= maxit || lucky) break;
        }
        for (int i = jend - 1; i >= 0; --i) {
            double sacc = g[i];
            for (int q = i + 1; q < jend; ++q) sacc -= H[(size_t)i * m + q] * y[q];
            y[i] = sacc / H[(size_t)i * m + i];
        }
        if (flexible) {
            for (int i = 0; i < jend; ++i) axpby(n, y[i], Z + (size_t)i * n, 1.0, x);
        } else {
            memset(w, 0, sizeof(double) * n);
            for (int i = 0; i < jend; ++i) axpby(n, y[i], V + (size_t)i * n, 1.0, w);
            int ps = or_pc_apply(s, w, t);
            if (ps) { st = ps; goto done; }
            axpby(n, 1.0, t, 1.0, x);
        }
    }
done:
    if (stats) {
        memcpy(w, b, sizeof(double) * n);
        or_spmv(s->nb, s->rp, s->ci, s->v, -1.0, x, 1.0, w);
        stats[0] = iters;
        stats[1] = cycles;
        stats[2] = or_norm2(n, w) / (bnorm > 0 ? bnorm : 1.0);
        stats[3] = (double)s->pc_applies;
    }
    free(V); free(Z); free(w); free(t); free(H); free(cs); free(sn); free(g); free(y);
    return st;
}

/* --------------------------------------------------------------- BiCGSTAB */

/* Right-preconditioned BiCGSTAB (van der Vorst):
 *   r = b - A x, rh = r, rho = alpha = omega = 1, v = p = 0; loop:
 *   rho' = <rh, r>; beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v);
 *   ph = M^{-1} p; v = A ph; alpha = rho' / <rh, v>; s = r - alpha v;
 *   if ||s|| <= tol: x += alpha ph, stop;
 *   sh = M^{-1} s; t = A sh; omega = <t,s>/<t,t>; x += alpha ph + omega sh;
 *   r = s - omega t; rho = rho'; stop if ||r|| <= tol.
 * |rho'|, |<rh,v>| or |omega| at or below btol (relative to the norms
 * involved) is a breakdown.  iters counts loop passes. */
int or_bicgstab(or_system *s, const double *b, double *x, double rtol, double btol, int maxit,
                double *stats) {
    int64_t n = 3 * (int64_t)s->nb;
    double *r = (double *)malloc(sizeof(double) * n), *rh = (double *)malloc(sizeof(double) * n);
    double *p = (double *)calloc(n, sizeof(double)), *v = (double *)calloc(n, sizeof(double));
    double *ph = (double *)malloc(sizeof(double) * n), *sh = (double *)malloc(sizeof(double) * n);
    double *sv = (double *)malloc(sizeof(double) * n), *t = (double *)malloc(sizeof(double) * n);
    double bnorm = or_norm2(n, b), tol = rtol * bnorm;
    memcpy(r, b, sizeof(double) * n);
    or_spmv(s->nb, s->rp, s->ci, s->v, -1.0, x, 1.0, r);
    memcpy(rh, r, sizeof(double) * n);
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0, st = OR_ENOCONV;
    s->pc_applies = 0;
    double rn = or_norm2(n, r);
    if (rn <= tol) st = OR_OK;
    double rhn = rn;
    while (st == OR_ENOCONV && it < maxit) {
        ++it;
        double rho1 = or_dot(n, rh, r);
        if (!isfinite(rho1)) { st = OR_ENAN; break; }
        if (fabs(rho1) <= btol * rhn * rn) { st = OR_EBREAKDOWN; break; }
        double beta = (rho1 / rho) * (alpha / omega);
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; ++q) p[q] = r[q] + beta * (p[q] - omega * v[q]);
        int ps = or_pc_apply(s, p, ph);
        if (ps) { st = ps; break; }
        or_spmv(s->nb, s->rp, s->ci, s->v, 1.0, ph, 0.0, v);
        double rv = or_dot(n, rh, v);
        if (fabs(rv) <= btol * rhn * or_norm2(n, v)) { st = OR_EBREAKDOWN; break; }
        alpha = rho1 / rv;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; ++q) sv[q] = r[q] - alpha * v[q];
        double sn = or_norm2(n, sv);
        if (sn <= tol) {
            axpby(n, alpha, ph, 1.0, x);
            st = OR_OK;
            break;
        }
        ps = or_pc_apply(s, sv, sh);
        if (ps) { st = ps; break; }
        or_spmv(s->nb, s->rp, s->ci, s->v, 1.0, sh, 0.0, t);
        double tt = or_dot(n, t, t);
        double ts = or_dot(n, t, sv);
        if (!(tt > 0.0)) { st = OR_EBREAKDOWN; break; }
        omega = ts / tt;
        if (fabs(omega) <= btol) { st = OR_EBREAKDOWN; break; }
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; ++q) {
            x[q] += alpha * ph[q] + omega * sh[q];
            r[q] = sv[q] - omega * t[q];
        }
        rho = rho1;
        rn = or_norm2(n, r);
        if (!isfinite(rn)) { st = OR_ENAN; break; }
        if (rn <= tol) st = OR_OK;
    }
    if (stats) {
        memcpy(r, b, sizeof(double) * n);
        or_spmv(s->nb, s->rp, s->ci, s->v, -1.0, x, 1.0, r);
        stats[0] = it;
        stats[1] = 0;
        stats[2] = or_norm2(n, r) / (bnorm > 0 ? bnorm : 1.0);
        stats[3] = (double)s->pc_applies;
    }
    free(r); free(rh); free(p); free(v); free(ph); free(sh); free(sv); free(t);
    return st;
}

/* ----------------------------------------------------- iterative refinement */

/* FP64 outer loop around inner solves on the float-rounded system `inner`:
 *   r = b - A64 x;  stop if ||r|| <= rtol ||b||;  solve inner d ~ r to
 *   inner_rtol (relative to ||r||) from d = 0;  x += d;  at most max_outer.
 * solver: 0 GMRES(m), 1 BiCGSTAB.  stats[0] = inner iterations summed,
 * stats[1] = outer steps, stats[2] = final true relative residual. */
int or_refine(or_system *outer, or_system *inner, const double *b, double *x, int solver, int m,
              double rtol, double inner_rtol, int max_outer, int maxit, double *stats) {
    int64_t n = 3 * (int64_t)outer->nb;
    double *r = (double *)malloc(sizeof(double) * n), *d = (double *)malloc(sizeof(double) * n);
    double bnorm = or_norm2(n, b);
    int outer_steps = 0, inner_total = 0, st = OR_ENOCONV;
    double rel = 1.0;
    for (;;) {
        memcpy(r, b, sizeof(double) * n);
        or_spmv(outer->nb, outer->rp, outer->ci, outer->v, -1.0, x, 1.0, r);
        double rn = or_norm2(n, r);
        rel = rn / (bnorm > 0 ? bnorm : 1.0);
        if (!isfinite(rn)) { st = OR_ENAN; break; }
        if (rn <= rtol * bnorm) { st = OR_OK; break; }
        if (outer_steps >= max_outer || inner_total >= maxit) { st = OR_ENOCONV; break; }
        ++outer_steps;
        memset(d, 0, sizeof(double) * n);
        double ist[4] = {0, 0, 0, 0};
        /* inner tolerance relative to ||r||: inner_rtol, or less strict on the last step,
           which only needs to bring ||r|| below rtol ||b|| (with a factor 2 of margin) */
        double itol = 0.5 * rtol * bnorm / rn;
        if (itol < inner_rtol) itol = inner_rtol;
        int is = (solver == 0) ? or_gmres(inner, r, d, m, itol, maxit - inner_total, 0, ist)
                               : or_bicgstab(inner, r, d, itol, 1e-30, maxit - inner_total, ist);
        inner_total += (int)ist[0];
        if (is != OR_OK && is != OR_ENOCONV) { st = is; break; }
        axpby(n, 1.0, d, 1.0, x);
    }
    if (stats) { stats[0] = inner_total; stats[1] = outer_steps; stats[2] = rel; stats[3] = 0; }
    free(r); free(d);
    return st;
}
