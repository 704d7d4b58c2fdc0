// CPR two-stage preconditioner (Section "CPR-like Preconditioners").
//
// Pressure stage: quasi-IMPES decoupling (named in the numerical experiments;
// diagonal reading: with D = A_cc, w_c = (1, -D01/D11, -D02/D22)), the
// restriction Pi_r f = (w_c . f_c)_c, and the pressure matrix
// (A_pp)_cn = sum_r w_c[r] A_cn[r][0] (the pressure column of the weighted
// block row), a seven-point scalar stencil.  It is solved approximately by
// one geometric-multigrid V-cycle standing in for the paper's AMG (Section
// "Algebraic Multigrid Methods": R = P^T, A_{l+1} = R A_l P, pre-smoother,
// residual, restriction, recursion, prolongation, post-smoother, exact
// coarsest solve):
//   * P is piecewise constant on 2x2x2 boxes (coarse dims ceil(d/2)), so the
//     Galerkin operator stays seven-point: entry (I, J) sums the fine
//     couplings from box I to box J, couplings inside a box add to I's centre;
//   * smoothing is red-black Gauss-Seidel, colour (i+j+k) mod 2, red then
//     black before the recursion and black then red after it;
//   * the coarsest level (at most gmg_max_coarse cells) is solved with its
//     explicit inverse, computed at setup from a partial-pivoting LU.
// Full stage (CPR-PF, two-stage multiplicative): x = Pi_p p; r = f - A x;
// x = x + ILU0^{-1} r, with Pi_p p = (p_c, 0, 0)_c.
//
// Stencil storage: a7[s][c] (slot-major, coalesced), slots -z, -y, -x,
// centre, +x, +y, +z; absent faces hold 0.
#include <algorithm>

#include "common.cuh"

namespace rsv {
namespace {

__device__ __forceinline__ bool gated(const int *done) { return done && *(volatile const int *)done; }

struct G3 {
    int nx, ny, nz;
    __host__ __device__ int64_t n() const { return (int64_t)nx * ny * nz; }
};

__device__ __forceinline__ void ijk(int64_t c, G3 g, int &i, int &j, int &k) {
    i = (int)(c % g.nx);
    j = (int)((c / g.nx) % g.ny);
    k = (int)(c / ((int64_t)g.nx * g.ny));
}

// The divisors of the smoother's index arithmetic, built on the host (Div32): ny and the
// colour slots of a grid row, ceil(nx / 2) (a level has < 2^31 cells).
struct G3Div {
    Div32 dy, dh;
    static G3Div of(const G3 &g) { return {Div32::of(g.ny), Div32::of((g.nx + 1) / 2)}; }
};


__constant__ int kDI[7] = {0, 0, -1, 0, 1, 0, 0};
__constant__ int kDJ[7] = {0, -1, 0, 0, 0, 1, 0};
__constant__ int kDK[7] = {-1, 0, 0, 0, 0, 0, 1};

__device__ __forceinline__ int slot_of(int di, int dj, int dk) {
    return dk < 0 ? 0 : dj < 0 ? 1 : di < 0 ? 2 : di > 0 ? 4 : dj > 0 ? 5 : dk > 0 ? 6 : 3;
}

// Quasi-IMPES weights and the pressure stencil of the block row of cell c.
template <typename Tv>
__global__ void qi_setup_kernel(G3 g, const int32_t *__restrict__ rp, const Tv *__restrict__ v, int decoupling,
                                const double *__restrict__ acc, double *__restrict__ w, double *__restrict__ a7,
                                int *status) {
    const int64_t n = g.n();
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    int i, j, k;
    ijk(c, g, i, j, k);
    const bool has[7] = {k > 0, j > 0, i > 0, true, i < g.nx - 1, j < g.ny - 1, k < g.nz - 1};
    int slot_pos[7], q = 0;
    for (int s = 0; s < 7; ++s) slot_pos[s] = has[s] ? q++ : -1;
    const Tv *dv = v + 9 * ((int64_t)rp[c] + slot_pos[3]);
    double d[9];
    if (decoupling == 2)  // true-IMPES: the cell's accumulation block instead of A's diagonal block
        for (int q = 0; q < 9; ++q) d[q] = acc[9 * c + q];
    else
        for (int q = 0; q < 9; ++q) d[q] = (double)dv[q];
    double w0, w1, w2;
    if (decoupling == 1 || decoupling == 2) {
        // ABF / true-IMPES: the first row of D^{-1} = adj(D) / det(D), from the cofactors of D's first column
        const double c0 = d[4] * d[8] - d[5] * d[7];
        const double det = d[0] * c0 + d[1] * (d[5] * d[6] - d[3] * d[8]) + d[2] * (d[3] * d[7] - d[4] * d[6]);
        if (!(fabs(det) > 1e-300)) {
            atomicCAS(status, 0, (int)RSV_ESINGULAR);
            return;
        }
        w0 = c0 / det;
        w1 = (d[2] * d[7] - d[1] * d[8]) / det;
        w2 = (d[1] * d[5] - d[2] * d[4]) / det;
    } else {
        // quasi-IMPES: keep the pressure equation, cancel the diagonal coupling of the other two
        if (!(fabs(d[4]) > 1e-300) || !(fabs(d[8]) > 1e-300)) {
            atomicCAS(status, 0, (int)RSV_ESINGULAR);
            return;
        }
        w0 = 1.0;
        w1 = -d[1] / d[4];
        w2 = -d[2] / d[8];
    }
    w[3 * c] = w0;
    w[3 * c + 1] = w1;
    w[3 * c + 2] = w2;
    for (int s = 0; s < 7; ++s) {
        double val = 0.0;
        if (has[s]) {
            const Tv *blk = v + 9 * ((int64_t)rp[c] + slot_pos[s]);
            val = w0 * (double)blk[0] + w1 * (double)blk[3] + w2 * (double)blk[6];
        }
        a7[(int64_t)s * n + c] = val;
    }
}

// Galerkin coarse operator P^T A P for piecewise-constant P: one thread per
// coarse cell sums the couplings of its children (children and slots in a
// fixed order, so the result is deterministic).
__global__ void gmg_coarsen_kernel(G3 f, const double *__restrict__ af, G3 cg, double *__restrict__ ac) {
    const int64_t nc = cg.n(), nf = f.n();
    const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (C >= nc) return;
    int I, J, K;
    ijk(C, cg, I, J, K);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                if (i >= f.nx || j >= f.ny || k >= f.nz) continue;
                const int64_t c = (int64_t)k * f.nx * f.ny + (int64_t)j * f.nx + i;
                for (int s = 0; s < 7; ++s) {
                    const int ii = i + kDI[s], jj = j + kDJ[s], kk = k + kDK[s];
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= f.nx || jj >= f.ny || kk >= f.nz) continue;
                    acc[slot_of(ii / 2 - I, jj / 2 - J, kk / 2 - K)] += af[(int64_t)s * nf + c];
                }
            }
    for (int s = 0; s < 7; ++s) ac[(int64_t)s * nc + C] = acc[s];
}

__global__ void cast_stencil(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// Dense matrix of the coarsest stencil, row-major n x n.
__global__ void coarse_dense_kernel(G3 g, const double *__restrict__ a7, double *__restrict__ M) {
    const int64_t n = g.n();
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int64_t q = 0; q < n; ++q) M[c * n + q] = 0.0;
    int i, j, k;
    ijk(c, g, i, j, k);
    for (int s = 0; s < 7; ++s) {
        const int ii = i + kDI[s], jj = j + kDJ[s], kk = k + kDK[s];
        if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
        M[c * n + (int64_t)kk * g.nx * g.ny + (int64_t)jj * g.nx + ii] += a7[(int64_t)s * n + c];
    }
}

// In-place LU with partial pivoting of the n x n matrix M (one CTA), then its
// inverse into Minv by solving for the unit vectors.  |pivot| <= 1e-300
// reports RSV_ESINGULAR.
__global__ void __launch_bounds__(1024) coarse_lu_kernel(int n, double *M, int *piv, int *status) {
    __shared__ double sval[32];
    __shared__ int sidx[32];
    __shared__ int spiv;
    for (int k = 0; k < n; ++k) {
        // pivot search in column k (max |M[i][k]|, smallest i on ties)
        double best = -1.0;
        int bi = k;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double a = fabs(M[(int64_t)i * n + k]);
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((threadIdx.x & 31) == 0) { sval[threadIdx.x >> 5] = best; sidx[threadIdx.x >> 5] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int p = k;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
                if (sval[q] > b || (sval[q] == b && sidx[q] < p)) { b = sval[q]; p = sidx[q]; }
            spiv = p;
            piv[k] = p;
            if (!(b > 1e-300)) atomicCAS(status, 0, (int)RSV_ESINGULAR);
        }
        __syncthreads();
        const int p = spiv;
        if (p != k)
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                const double t = M[(int64_t)k * n + q];
                M[(int64_t)k * n + q] = M[(int64_t)p * n + q];
                M[(int64_t)p * n + q] = t;
            }
        __syncthreads();
        const double pk = M[(int64_t)k * n + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) M[(int64_t)i * n + k] /= pk;
        __syncthreads();
        const int m = n - k - 1;
        for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += blockDim.x) {
            const int i = k + 1 + (int)(t / m), q = k + 1 + (int)(t % m);
            M[(int64_t)i * n + q] -= M[(int64_t)i * n + k] * M[(int64_t)k * n + q];
        }
        __syncthreads();
    }
}

// Column j of the inverse: solve (LU) x = P e_j.  One CTA per column.
__global__ void coarse_inverse_kernel(int n, const double *__restrict__ LU, const int *__restrict__ piv,
                                      double *__restrict__ Minv, double *__restrict__ work) {
    const int j = blockIdx.x;
    double *x = work + (int64_t)j * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < n; ++k)
            if (piv[k] != k) {
                const double t = x[k];
                x[k] = x[piv[k]];
                x[piv[k]] = t;
            }
    __syncthreads();
    for (int k = 0; k < n; ++k) {  // unit lower triangle
        const double xk = x[k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) x[i] -= LU[(int64_t)i * n + k] * xk;
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {  // upper triangle
        if (threadIdx.x == 0) x[k] /= LU[(int64_t)k * n + k];
        __syncthreads();
        const double xk = x[k];
        for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] -= LU[(int64_t)i * n + k] * xk;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) Minv[(int64_t)i * n + j] = x[i];
}

// x = Minv b (one warp per row), b and x in T, arithmetic in FP64.
template <typename T>
__global__ void coarse_apply_kernel(int n, const double *__restrict__ Minv, const T *__restrict__ b, T *__restrict__ x,
                                    const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (gated(done)) return;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int q = lane; q < n; q += 32) s += Minv[(int64_t)row * n + q] * (double)b[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = (T)s;
}

// Colour-split position of the cell (2 h + parity, j, k) of colour `colour` in grid row
// row = j + ny k: the row's red cells first (i ascending), then its black cells.  A row
// starting with a red cell ((j + k) even) holds ceil(nx / 2) red cells, else floor(nx / 2).
__device__ __forceinline__ int64_t split_pos(G3 g, int64_t row, int j, int k, int h, int colour) {
    const int nred = (g.nx + 1 - ((j + k) & 1)) >> 1;
    return row * g.nx + (colour == 0 ? h : nred + h);
}

// a7s[s][split_pos(c)] = a7[s][c] (converted to T).
template <typename T>
__global__ void split_stencil_kernel(G3 g, const double *__restrict__ a7, T *__restrict__ a7s) {
    const int64_t n = g.n();
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    int i, j, k;
    ijk(c, g, i, j, k);
    const int64_t ps = split_pos(g, c / g.nx, j, k, i >> 1, (i + j + k) & 1);
    for (int s = 0; s < 7; ++s) a7s[(int64_t)s * n + ps] = (T)a7[(int64_t)s * n + c];
}

// One red-black Gauss-Seidel half sweep over the cells of colour (i+j+k) mod 2;
// one thread per cell of that colour (a row of nx cells holds ceil(nx/2) or
// floor(nx/2) of them).  Cells of one colour couple only to the other colour,
// so the update x_c = (b_c - sum_n a_cn x_n) / a_cc reads only cells this
// launch does not write.  MODE selects what the neighbours hold:
//   0  x as stored;
//   1  zero (the first half sweep of a V-cycle level from a zero guess:
//      x_c = b_c / a_cc, and x need not be cleared first);
//   2  x + P xc (the first half sweep after the coarse correction: the
//      prolongation x += P xc is applied to the neighbours on the fly; this
//      colour's own cells are overwritten, so the correction need not be
//      stored for them, and the other colour's cells are overwritten by the
//      next half sweep, which reads only this colour).
// Each variant rounds exactly as the separate zeroing / prolongation kernels
// followed by the plain half sweep.
//
// The coefficients come from a colour-split copy a7s (see split_pos): the cells
// of one colour in a grid row are contiguous there, so a half sweep reads
// only its own colour's coefficients, coalesced.
// Each thread takes CELLS cells of the colour, blockDim.x colour slots apart (coalesced per
// slot), and issues all their loads before any store: same-colour cells never read one
// another.  On large levels the loads in flight per thread, not bandwidth, bound the
// one-cell form (finest level of 256x256x128: 47 us per half sweep, 38 us with four cells);
// small levels and the prolongating sweep (MODE 2) keep one cell per thread.
template <typename T, int MODE, int CELLS>
__global__ void rbgs_kernel(G3 g, G3Div gd, const T *__restrict__ a7s, const T *__restrict__ b, T *__restrict__ x,
                            int colour, const T *__restrict__ xc, G3 cg, const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (gated(done)) return;
    const int64_t n = g.n();
    const int half = (g.nx + 1) >> 1;
    const int rows = g.ny * g.nz;
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    T res[CELLS];
    int64_t cell[CELLS];
#pragma unroll
    for (int u = 0; u < CELLS; ++u) {
        cell[u] = -1;
        const int q = (blockIdx.x * CELLS + u) * blockDim.x + threadIdx.x;
        const int row = gd.dh(q);  // row = j + ny k
        if (row >= rows) continue;
        const int k = gd.dy(row), j = row - k * g.ny;
        const int h = q - row * half;
        const int i = 2 * h + ((colour + j + k) & 1);
        if (i >= g.nx) continue;
        const int64_t c = (int64_t)row * g.nx + i;
        const T *a7 = a7s + split_pos(g, row, j, k, h, colour);  // slot s at a7[s * n]
        T s = b[c];
        if (MODE != 1) {
            auto nbr = [&](int64_t o, int ii, int jj, int kk) -> T {
                T v = x[o];
                if (MODE == 2) v += xc[(int64_t)(kk >> 1) * cg.nx * cg.ny + (int64_t)(jj >> 1) * cg.nx + (ii >> 1)];
                return v;
            };
            if (k > 0) s -= a7[0 * n] * nbr(c - sz, i, j, k - 1);
            if (j > 0) s -= a7[1 * n] * nbr(c - sy, i, j - 1, k);
            if (i > 0) s -= a7[2 * n] * nbr(c - 1, i - 1, j, k);
            if (i < g.nx - 1) s -= a7[4 * n] * nbr(c + 1, i + 1, j, k);
            if (j < g.ny - 1) s -= a7[5 * n] * nbr(c + sy, i, j + 1, k);
            if (k < g.nz - 1) s -= a7[6 * n] * nbr(c + sz, i, j, k + 1);
        }
        res[u] = s / a7[3 * n];
        cell[u] = c;
    }
#pragma unroll
    for (int u = 0; u < CELLS; ++u)
        if (cell[u] >= 0) x[cell[u]] = res[u];
}

// b_coarse[C] = sum over the children f of C of (b_f - (A x)_f): residual and
// restriction R = P^T fused.
template <typename T>
__global__ void residual_restrict_kernel(G3 f, const T *__restrict__ a7, const T *__restrict__ b,
                                         const T *__restrict__ x, G3 cg, T *__restrict__ bc, const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (gated(done)) return;
    const int64_t nc = cg.n(), n = f.n();
    const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (C >= nc) return;
    int I, J, K;
    ijk(C, cg, I, J, K);
    const int64_t sy = f.nx, sz = (int64_t)f.nx * f.ny;
    T acc = T(0);
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                if (i >= f.nx || j >= f.ny || k >= f.nz) continue;
                const int64_t c = (int64_t)k * sz + (int64_t)j * sy + i;
                T r = b[c] - a7[3 * n + c] * x[c];
                if (k > 0) r -= a7[0 * n + c] * x[c - sz];
                if (j > 0) r -= a7[1 * n + c] * x[c - sy];
                if (i > 0) r -= a7[2 * n + c] * x[c - 1];
                if (i < f.nx - 1) r -= a7[4 * n + c] * x[c + 1];
                if (j < f.ny - 1) r -= a7[5 * n + c] * x[c + sy];
                if (k < f.nz - 1) r -= a7[6 * n + c] * x[c + sz];
                acc += r;
            }
    bc[C] = acc;
}

// x_fine += P x_coarse (injection of the box value).
template <typename T>
__global__ void prolong_add_kernel(G3 f, const T *__restrict__ xc, G3 cg, T *__restrict__ x, const int *done) {
    if (gated(done)) return;
    const int64_t n = f.n();
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    int i, j, k;
    ijk(c, f, i, j, k);
    x[c] += xc[(int64_t)(k / 2) * cg.nx * cg.ny + (int64_t)(j / 2) * cg.nx + i / 2];
}

// x += P xc on a large level, four consecutive cells of a grid row per thread (all loads
// before the stores).  dq divides by the row's quads, ceil(nx / 4); dy by ny.  Each cell's
// sum is the one prolong_add_kernel forms.
template <typename T>
__global__ void prolong_add_rows(G3 f, Div32 dq, Div32 dy, const T *__restrict__ xc, G3 cg, T *__restrict__ x,
                                 const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (gated(done)) return;
    const int quads = (f.nx + 3) >> 2;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = dq(q);
    if (row >= f.ny * f.nz) return;
    const int k = dy(row), j = row - k * f.ny, i0 = 4 * (q - row * quads);
    T *xr = x + (int64_t)row * f.nx;
    const T *cr = xc + (int64_t)(k >> 1) * cg.nx * cg.ny + (int64_t)(j >> 1) * cg.nx;
    if constexpr (sizeof(T) == 4) {
        if ((f.nx & 3) == 0 && (((uintptr_t)x) & 15) == 0) {  // one 16-byte access per quad
            float4 v = *reinterpret_cast<const float4 *>(xr + i0);
            const T p0 = cr[i0 >> 1], p1 = cr[(i0 >> 1) + 1];
            v.x += p0;
            v.y += p0;
            v.z += p1;
            v.w += p1;
            *reinterpret_cast<float4 *>(xr + i0) = v;
            return;
        }
    }
    T v[4], p[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (i0 + u < f.nx) {
            v[u] = xr[i0 + u];
            p[u] = cr[(i0 + u) >> 1];
        }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (i0 + u < f.nx) xr[i0 + u] = v[u] + p[u];
}

template <typename T>
__global__ void zero_kernel(int64_t n, T *x, const int *done) {
    if (gated(done)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = T(0);
}

// p_c = w_c . f_c
template <typename T>
__global__ void restrict_pressure_kernel(int64_t nb, const T *__restrict__ w, const T *__restrict__ f,
                                         T *__restrict__ p, const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (gated(done)) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    p[c] = w[3 * c] * f[3 * c] + w[3 * c + 1] * f[3 * c + 1] + w[3 * c + 2] * f[3 * c + 2];
}

// The same for FP32 with 16-byte accesses: four cells per thread (three float4 loads of w and
// of f, one float4 store), each cell's products and sums written as above.  Needs nb % 4 == 0
// and 16-byte aligned w, f and p.
__global__ void restrict_pressure_v4(int64_t nb4, const float4 *__restrict__ w, const float4 *__restrict__ f,
                                     float4 *__restrict__ p, const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (gated(done)) return;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nb4) return;
    const float4 w0 = w[3 * t], w1 = w[3 * t + 1], w2 = w[3 * t + 2];
    const float4 f0 = f[3 * t], f1 = f[3 * t + 1], f2 = f[3 * t + 2];
    float4 o;
    o.x = w0.x * f0.x + w0.y * f0.y + w0.z * f0.z;
    o.y = w0.w * f0.w + w1.x * f1.x + w1.y * f1.y;
    o.z = w1.z * f1.z + w1.w * f1.w + w2.x * f2.x;
    o.w = w2.y * f2.y + w2.z * f2.z + w2.w * f2.w;
    p[t] = o;
}

// x_c = (p_c, 0, 0) and r = f (the copy the stage-two residual starts from)
template <typename T>
__global__ void prolong_pressure_kernel(int64_t nb, const T *__restrict__ p, const T *__restrict__ f,
                                        T *__restrict__ x, T *__restrict__ r, const int *done) {
    if (gated(done)) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    x[3 * c] = p[c];
    x[3 * c + 1] = T(0);
    x[3 * c + 2] = T(0);
    r[3 * c] = f[3 * c];
    r[3 * c + 1] = f[3 * c + 1];
    r[3 * c + 2] = f[3 * c + 2];
}

// The pressure column of every block, apc[3 q + e] = A_q[e][0] (in the solver's precision).
template <typename Tv, typename T>
__global__ void pressure_columns_kernel(int64_t nnzb, const Tv *__restrict__ v, T *__restrict__ apc) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnzb; q += (int64_t)gridDim.x * blockDim.x) {
        apc[3 * q] = (T)v[9 * q];
        apc[3 * q + 1] = (T)v[9 * q + 3];
        apc[3 * q + 2] = (T)v[9 * q + 6];
    }
}

// x_c += (p_c, 0, 0): a pressure-stage correction added to the iterate
template <typename T>
__global__ void prolong_add_pressure_kernel(int64_t nb, const T *__restrict__ p, T *__restrict__ x, const int *done) {
    if (gated(done)) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    x[3 * c] += p[c];
}

template <typename T>
__global__ void add_kernel(int64_t n, const T *__restrict__ z, T *__restrict__ x, const int *done) {
    if (gated(done)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += z[i];
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

void free_cpr(Cpr *P) {
    amg_free(P);
    for (int l = 0; l < kMaxLevels; ++l)
        for (void *p : {(void *)P->a7[l], P->a7f[l], P->a7s[l], P->x[l], P->b[l]})
            if (p) cudaFree(p);
    for (void *p : {(void *)P->w64, P->w, (void *)P->minv, (void *)P->dense, (void *)P->piv, (void *)P->work,
                    P->r, P->z, P->xp, P->apc})
        if (p) cudaFree(p);
    *P = Cpr();
}

cudaError_t cpr_setup(const rsv_mat *A, bool mixed, int max_levels, int max_coarse, int sweeps, int decoupling,
                      const double *acc, int coarsening, Cpr *P, int *status) {
    cudaStream_t st = A->stream;
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    amg_free(P);
    if (coarsening == 1) max_levels = 1;  // the geometric part keeps only the finest level
    // level sizes: halve (ceil) each dimension while the level has more than max_coarse cells
    int dims[kMaxLevels][3];
    G3 g{A->nx, A->ny, A->nz};
    int nl = 0;
    dims[nl][0] = g.nx, dims[nl][1] = g.ny, dims[nl][2] = g.nz;
    ++nl;
    max_levels = std::min(std::max(max_levels, 1), kMaxLevels);
    while (nl < max_levels && g.n() > max_coarse) {
        g = G3{(g.nx + 1) / 2, (g.ny + 1) / 2, (g.nz + 1) / 2};
        dims[nl][0] = g.nx, dims[nl][1] = g.ny, dims[nl][2] = g.nz;
        ++nl;
    }
    // a new setup of the same hierarchy (the usual case: new values, same grid) reuses the buffers
    bool same = P->w64 && P->mixed == mixed && P->nlev == nl;
    for (int l = 0; same && l < nl; ++l)
        for (int d = 0; d < 3; ++d) same = same && P->dims[l][d] == dims[l][d];
    if (!same) free_cpr(P);
    P->mixed = mixed;
    P->sweeps = sweeps;
    for (int l = 0; l < nl; ++l)
        for (int d = 0; d < 3; ++d) P->dims[l][d] = dims[l][d];
    P->nlev = nl;
    const int64_t nb = A->nb;
    const int nc = (int)g.n();
    P->ncoarse = nc;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess && !same) e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    };
    alloc((void **)&P->w64, sizeof(double) * 3 * nb);
    alloc(&P->w, es * 3 * nb);
    for (int l = 0; l < nl; ++l) {
        const int64_t n = (int64_t)P->dims[l][0] * P->dims[l][1] * P->dims[l][2];
        alloc((void **)&P->a7[l], sizeof(double) * 7 * n);
        if (mixed) alloc(&P->a7f[l], sizeof(float) * 7 * n);
        if (l + 1 < nl) alloc(&P->a7s[l], es * 7 * n);
        alloc(&P->x[l], es * n);
        alloc(&P->b[l], es * n);
    }
    const int64_t ncd = coarsening == 1 ? 1 : nc;  // the algebraic hierarchy keeps its own coarsest inverse
    alloc((void **)&P->dense, sizeof(double) * ncd * ncd);
    alloc((void **)&P->minv, sizeof(double) * ncd * ncd);
    alloc((void **)&P->work, sizeof(double) * ncd * ncd);
    alloc((void **)&P->piv, sizeof(int) * ncd);
    alloc(&P->r, es * 3 * nb);
    alloc(&P->z, es * 3 * nb);
    alloc(&P->xp, es * 3 * nb);
    alloc(&P->apc, es * 3 * (size_t)A->nnzb + 64);  // tail room: the residual kernels stage whole 16-byte units
    if (e != cudaSuccess) return e;
    G3 g0{A->nx, A->ny, A->nz};
    count_launches(1);
    if (mixed)
        qi_setup_kernel<float><<<blocks(nb), 256, 0, st>>>(g0, A->d_rp, A->d_v32, decoupling, acc, P->w64, P->a7[0],
                                                           status);
    else
        qi_setup_kernel<double><<<blocks(nb), 256, 0, st>>>(g0, A->d_rp, A->d_v, decoupling, acc, P->w64, P->a7[0],
                                                            status);
    for (int l = 0; l + 1 < nl; ++l) {
        G3 f{P->dims[l][0], P->dims[l][1], P->dims[l][2]}, c{P->dims[l + 1][0], P->dims[l + 1][1], P->dims[l + 1][2]};
        count_launches(1);
        gmg_coarsen_kernel<<<blocks(c.n()), 256, 0, st>>>(f, P->a7[l], c, P->a7[l + 1]);
    }
    if (coarsening != 1) {
        G3 gc{P->dims[nl - 1][0], P->dims[nl - 1][1], P->dims[nl - 1][2]};
        count_launches(3);
        coarse_dense_kernel<<<blocks(nc), 256, 0, st>>>(gc, P->a7[nl - 1], P->dense);
        coarse_lu_kernel<<<1, 1024, 0, st>>>(nc, P->dense, P->piv, status);
        coarse_inverse_kernel<<<nc, 128, 0, st>>>(nc, P->dense, P->piv, P->minv, P->work);
    }
    const unsigned pcb = (unsigned)std::min<int64_t>(blocks(A->nnzb), 152 * 32);
    count_launches(1);
    if (mixed)
        pressure_columns_kernel<float, float><<<pcb, 256, 0, st>>>(A->nnzb, A->d_v32, (float *)P->apc);
    else
        pressure_columns_kernel<double, double><<<pcb, 256, 0, st>>>(A->nnzb, A->d_v, (double *)P->apc);
    for (int l = 0; l + 1 < nl; ++l) {  // the smoothed levels' colour-split coefficients
        G3 g{P->dims[l][0], P->dims[l][1], P->dims[l][2]};
        count_launches(1);
        if (mixed)
            split_stencil_kernel<float><<<blocks(g.n()), 256, 0, st>>>(g, P->a7[l], (float *)P->a7s[l]);
        else
            split_stencil_kernel<double><<<blocks(g.n()), 256, 0, st>>>(g, P->a7[l], (double *)P->a7s[l]);
    }
    if (mixed) {
        count_launches(1 + nl);
        cast_stencil<<<blocks(3 * nb), 256, 0, st>>>(3 * nb, P->w64, (float *)P->w);
        for (int l = 0; l < nl; ++l) {
            const int64_t n = (int64_t)P->dims[l][0] * P->dims[l][1] * P->dims[l][2];
            cast_stencil<<<blocks(7 * n), 256, 0, st>>>(7 * n, P->a7[l], (float *)P->a7f[l]);
        }
    } else {
        e = cudaMemcpyAsync(P->w, P->w64, sizeof(double) * 3 * nb, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// One V-cycle on level l from a zero initial guess: x[l] = V(b[l]).
template <typename T>
static cudaError_t vcycle(const Cpr &P, int l, cudaStream_t st, const int *done) {
    if (l == 0 && P.amg) return amg_vcycle<T>(P, st, done);
    const T *a7 = P.mixed ? (const T *)P.a7f[l] : (const T *)P.a7[l];
    const T *a7s = (const T *)P.a7s[l];  // colour-split copy for the smoother
    T *x = (T *)P.x[l], *b = (T *)P.b[l];
    G3 g{P.dims[l][0], P.dims[l][1], P.dims[l][2]};
    const int64_t n = g.n();
    // The cycle's kernels are launched as programmatic dependents (launch_pdl): each waits for
    // its predecessor on the device, so the launch latency of most levels' small kernels overlaps
    // the kernel before.
    if (l == P.nlev - 1) {
        count_launches(1);
        return launch_pdl(coarse_apply_kernel<T>, dim3(blocks(n * 32)), dim3(256), 0, st, (int)n, P.minv, b, x,
                          done);
    }
    G3 c{P.dims[l + 1][0], P.dims[l + 1][1], P.dims[l + 1][2]};
    const T *xc = (const T *)P.x[l + 1];
    const int64_t slots = (int64_t)((g.nx + 1) / 2) * g.ny * g.nz;  // colour slots of a half sweep
    const bool wide = slots >= (1 << 20);                             // four cells per thread
    const dim3 hb(blocks(slots)), hb4(blocks(slots, 256 * 4)), t256(256);
    const G3Div gd = G3Div::of(g);
    cudaError_t e = cudaSuccess;
    auto sweep = [&](auto kern, dim3 grid, int colour) {
        if (e == cudaSuccess) e = launch_pdl(kern, grid, t256, 0, st, g, gd, a7s, b, x, colour, xc, c, done);
    };
    auto half_sweep0 = [&](int colour) {
        if (wide)
            sweep(rbgs_kernel<T, 0, 4>, hb4, colour);
        else
            sweep(rbgs_kernel<T, 0, 1>, hb, colour);
    };
    // pre-smoothing from x = 0: red, black, `sweeps` times (the first red half sweep reads no neighbour)
    count_launches(P.sweeps > 0 ? 2 * P.sweeps : 1);
    if (P.sweeps == 0) zero_kernel<T><<<blocks(n), 256, 0, st>>>(n, x, done);
    for (int s = 0; s < P.sweeps; ++s) {
        if (s > 0)
            half_sweep0(0);
        else if (wide)
            sweep(rbgs_kernel<T, 1, 4>, hb4, 0);
        else
            sweep(rbgs_kernel<T, 1, 1>, hb, 0);
        half_sweep0(1);
    }
    count_launches(1);
    if (e == cudaSuccess)
        e = launch_pdl(residual_restrict_kernel<T>, dim3(blocks(c.n())), t256, 0, st, g, a7, b, x, c, (T *)P.b[l + 1],
                       done);
    if (e == cudaSuccess) e = vcycle<T>(P, l + 1, st, done);
    if (e != cudaSuccess) return e;
    // coarse correction x += P xc and post-smoothing black, red, `sweeps` times (the first black half
    // sweep applies the correction to the red values it reads)
    count_launches(P.sweeps > 0 ? 2 * P.sweeps : 1);
    if (P.sweeps == 0) prolong_add_kernel<T><<<blocks(n), 256, 0, st>>>(g, xc, c, x, done);
    for (int s = 0; s < P.sweeps; ++s) {
        if (s > 0) {
            half_sweep0(1);
        } else if (wide) {
            // on a large level the correction pass and a four-cell sweep beat the one-cell
            // prolongating sweep (finest level of 256x256x128: 68 us for MODE 2)
            count_launches(1);
            const int64_t quads = (int64_t)((g.nx + 3) / 4) * g.ny * g.nz;
            if (e == cudaSuccess)
                e = launch_pdl(prolong_add_rows<T>, dim3(blocks(quads)), t256, 0, st, g, Div32::of((g.nx + 3) / 4),
                               Div32::of(g.ny), xc, c, x, done);
            half_sweep0(1);
        } else {
            sweep(rbgs_kernel<T, 2, 1>, hb, 1);
        }
        half_sweep0(0);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Stage one, first half: the restricted right-hand side P.b[0] = Pi_r f.
template <typename T>
cudaError_t cpr_restrict(const rsv_mat *A, const Cpr &P, const T *f, const int *done) {
    count_launches(1);
    const bool v4 = sizeof(T) == 4 && A->nb % 4 == 0 && ((((uintptr_t)P.w) | ((uintptr_t)f) | ((uintptr_t)P.b[0])) & 15) == 0;
    if (v4)
        return launch_pdl(restrict_pressure_v4, dim3(blocks(A->nb / 4)), dim3(256), 0, A->stream, A->nb / 4,
                          (const float4 *)P.w, (const float4 *)f, (float4 *)P.b[0], done);
    return launch_pdl(restrict_pressure_kernel<T>, dim3(blocks(A->nb)), dim3(256), 0, A->stream, A->nb,
                      (const T *)P.w, f, (T *)P.b[0], done);
}

// The pressure solve P.x[0] = V-cycle(P.b[0]); kernels skip when *gate != 0.
template <typename T>
cudaError_t cpr_pressure_vcycle(const rsv_mat *A, const Cpr &P, const int *gate) {
    return vcycle<T>(P, 0, A->stream, gate);
}

// Stage one's prolongation x = Pi_p P.x[0], then stage two: x += ILU0^{-1}(f - A x).  Fused:
// r = f - A Pi_p p from the pressure columns alone, then x = ILU0^{-1} r + Pi_p p (the same
// sums, in the same order, as forming x = Pi_p p, r = f - A x and x += ILU0^{-1} r).
template <typename T>
cudaError_t cpr_finish(const rsv_mat *A, const Cpr &P, const IluTiles &tiles, const T *f, T *x, const int *done,
                       int *status, unsigned long long timeout_ns) {
    T *r = (T *)P.r;
    const T *p = (const T *)P.x[0];
    cudaError_t e = launch_pressure_residual<T>(A, (const T *)P.apc, p, f, r, done, status, timeout_ns);
    if (e != cudaSuccess) return e;
    // x = ILU0^{-1} r, and x_c[0] += p_c as the backward sweep stores x: p_c rides in the pad slot
    // of the sweeps' tile-order vectors, so no step of the sweeps waits on a load of p
    return launch_ilu_apply_tiles<T>(A, tiles, r, x, done, status, timeout_ns, p);
}

template <typename T>
cudaError_t cpr_apply(const rsv_mat *A, const Cpr &P, const IluTiles &tiles, const T *f, T *x, const int *done,
                      int *status, unsigned long long timeout_ns) {
    cudaError_t e = cpr_restrict<T>(A, P, f, done);
    if (e == cudaSuccess) e = vcycle<T>(P, 0, A->stream, done);
    if (e == cudaSuccess) e = cpr_finish<T>(A, P, tiles, f, x, done, status, timeout_ns);
    return e;
}

// The CPR orders of Section "CPR-like preconditioners" (Algorithms CPR-FP, CPR-PF,
// CPR-FPF, CPR-FFPF) as a string of stages.  The first stage writes x from f;
// every later stage forms r = f - A x (a copy of f and one SpMV) and adds its
// correction: F adds ILU0^{-1} r, P adds Pi_p V-cycle(Pi_r r).
template <typename T>
cudaError_t cpr_apply_order(const rsv_mat *A, const Cpr &P, const IluTiles &tiles, const char *stages, const T *f,
                            T *x, const int *done, int *status, unsigned long long timeout_ns) {
    cudaStream_t st = A->stream;
    const int64_t nb = A->nb;
    T *r = (T *)P.r, *z = (T *)P.z;
    cudaError_t e = cudaSuccess;
    for (int q = 0; stages[q] && e == cudaSuccess; ++q) {
        const T *src = f;
        if (q > 0) {
            e = cudaMemcpyAsync(r, f, sizeof(T) * 3 * nb, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = (sizeof(T) == 8) ? launch_spmv_f64(A, -1.0, (const double *)x, 1.0, (double *)r, done, status, timeout_ns)
                                     : launch_spmv_f32(A, -1.0f, (const float *)x, 1.0f, (float *)r, done, status,
                                                       timeout_ns);
            src = r;
        }
        if (e != cudaSuccess) break;
        if (stages[q] == 'F') {
            e = launch_ilu_apply_tiles<T>(A, tiles, src, q == 0 ? x : z, done, status, timeout_ns);
            if (e == cudaSuccess && q > 0) {
                count_launches(1);
                add_kernel<T><<<blocks(3 * nb), 256, 0, st>>>(3 * nb, z, x, done);
                e = cudaGetLastError();
            }
        } else {
            e = cpr_restrict<T>(A, P, src, done);
            if (e == cudaSuccess) e = vcycle<T>(P, 0, st, done);
            if (e == cudaSuccess) {
                count_launches(1);
                if (q == 0)
                    prolong_pressure_kernel<T><<<blocks(nb), 256, 0, st>>>(nb, (const T *)P.x[0], f, x, r, done);
                else
                    prolong_add_pressure_kernel<T><<<blocks(nb), 256, 0, st>>>(nb, (const T *)P.x[0], x, done);
                e = cudaGetLastError();
            }
        }
    }
    return e;
}

template <typename T>
cudaError_t cpr_vcycle(const rsv_mat *A, const Cpr &P, const T *b, T *x) {
    const int64_t n = A->nb;
    cudaError_t e = cudaMemcpyAsync(P.b[0], b, sizeof(T) * n, cudaMemcpyDeviceToDevice, A->stream);
    if (e == cudaSuccess) e = vcycle<T>(P, 0, A->stream, nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, P.x[0], sizeof(T) * n, cudaMemcpyDeviceToDevice, A->stream);
    return e;
}

template cudaError_t cpr_apply<double>(const rsv_mat *, const Cpr &, const IluTiles &, const double *, double *,
                                       const int *, int *, unsigned long long);
template cudaError_t cpr_apply<float>(const rsv_mat *, const Cpr &, const IluTiles &, const float *, float *,
                                      const int *, int *, unsigned long long);
template cudaError_t cpr_apply_order<double>(const rsv_mat *, const Cpr &, const IluTiles &, const char *,
                                             const double *, double *, const int *, int *, unsigned long long);
template cudaError_t cpr_apply_order<float>(const rsv_mat *, const Cpr &, const IluTiles &, const char *,
                                            const float *, float *, const int *, int *, unsigned long long);
template cudaError_t cpr_vcycle<double>(const rsv_mat *, const Cpr &, const double *, double *);
template cudaError_t cpr_restrict<double>(const rsv_mat *, const Cpr &, const double *, const int *);
template cudaError_t cpr_pressure_vcycle<double>(const rsv_mat *, const Cpr &, const int *);
template cudaError_t cpr_finish<double>(const rsv_mat *, const Cpr &, const IluTiles &, const double *, double *,
                                        const int *, int *, unsigned long long);
template cudaError_t cpr_vcycle<float>(const rsv_mat *, const Cpr &, const float *, float *);

}  // namespace rsv
