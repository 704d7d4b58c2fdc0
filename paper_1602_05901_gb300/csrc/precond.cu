// Block-Jacobi and block ILU(0) preconditioners on the seven-point 3x3-block
// Jacobian.
//
// Block ILU(0) (Section "Restricted Additive Schwarz Method": LU x = b is
// solved as L y = b, U x = y; ILU(0) is the default local solver).  For a
// seven-point pattern the no-fill factor only changes diagonal blocks (the
// grid graph has no triangles), so it is stored as D_c^{-1} with
//     D_c = A_cc - sum_{l in lower(c)} A_cl D_l^{-1} A_lc,
// and applied as M = (D + L_A) D^{-1} (D + U_A):
//     forward  y_c = D_c^{-1} (r_c - sum_{l < c} A_cl y_l)
//     backward z_c = y_c - D_c^{-1} sum_{u > c} A_cu z_u.
// Every lower neighbour of cell (i,j,k) lies on hyperplane i+j+k-1, so all
// cells of one hyperplane are independent; planes run in order (forward) or
// reverse order (backward).  This is a legal schedule of the natural-order
// recurrence, not a reordering: results equal the sequential factor up to
// rounding.
#include <algorithm>

#include "common.cuh"

namespace rsv {
namespace {

struct Dims {
    int nx, ny, nz;
};

__device__ __forceinline__ bool inv3(const double *a, double *o) {
    const double c00 = a[4] * a[8] - a[5] * a[7];
    const double c01 = a[5] * a[6] - a[3] * a[8];
    const double c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (!(fabs(det) > 1e-300)) return false;
    const double id = 1.0 / det;
    o[0] = c00 * id;
    o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
    o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    o[3] = c01 * id;
    o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
    o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    o[6] = c02 * id;
    o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
    o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
    return true;
}

__device__ __forceinline__ void mv3(const double *a, const double *x, double *y) {
    y[0] = a[0] * x[0] + a[1] * x[1] + a[2] * x[2];
    y[1] = a[3] * x[0] + a[4] * x[1] + a[5] * x[2];
    y[2] = a[6] * x[0] + a[7] * x[1] + a[8] * x[2];
}

__device__ __forceinline__ void mm3(const double *a, const double *b, double *c) {
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int f = 0; f < 3; ++f) c[3 * e + f] = a[3 * e] * b[f] + a[3 * e + 1] * b[3 + f] + a[3 * e + 2] * b[6 + f];
}

__device__ __forceinline__ void load9(const double *p, double *o) {
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] = p[q];
}

// Position of the blocks of row c inside the BSR row (columns ascending:
// -z, -y, -x, self, +x, +y, +z, absent faces skipped).
struct RowSlots {
    int mz, my, mx, d, px, py, pz;  // -1 when the face is absent
};

__device__ __forceinline__ RowSlots row_slots(int c, Dims g) {
    const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    RowSlots s;
    int q = 0;
    s.mz = (k > 0) ? q++ : -1;
    s.my = (j > 0) ? q++ : -1;
    s.mx = (i > 0) ? q++ : -1;
    s.d = q++;
    s.px = (i < g.nx - 1) ? q++ : -1;
    s.py = (j < g.ny - 1) ? q++ : -1;
    s.pz = (k < g.nz - 1) ? q++ : -1;
    return s;
}

__global__ void bj_setup_kernel(int64_t nb, Dims g, const int32_t *__restrict__ rp, const double *__restrict__ v,
                                double *__restrict__ dinv, int *status) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    const RowSlots s = row_slots((int)c, g);
    double a[9];
    load9(v + 9 * (int64_t)(rp[c] + s.d), a);
    if (!inv3(a, dinv + 9 * c)) atomicCAS(status, 0, (int)RSV_ESINGULAR);
}

__global__ void bj_apply_kernel(int64_t nb, const double *__restrict__ dinv, const double *__restrict__ r,
                                double *__restrict__ z, const int *done) {
    if (done && *(volatile const int *)done) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    double d[9], x[3], y[3];
    load9(dinv + 9 * c, d);
    x[0] = r[3 * c];
    x[1] = r[3 * c + 1];
    x[2] = r[3 * c + 2];
    mv3(d, x, y);
    z[3 * c] = y[0];
    z[3 * c + 1] = y[1];
    z[3 * c + 2] = y[2];
}

// D_c = A_cc - sum_{l lower} (A_cl D_l^{-1}) A_lc, lower neighbours in
// ascending column order (-z, -y, -x).
__global__ void ilu_factor_plane(Dims g, const int32_t *__restrict__ rp, const double *__restrict__ v,
                                 const int32_t *__restrict__ cells, int p0, int p1, double *dinv, int *status) {
    const int t = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p1) return;
    const int c = cells[t];
    const RowSlots s = row_slots(c, g);
    const int64_t base = rp[c];
    double D[9];
    load9(v + 9 * (base + s.d), D);
    const int lower[3] = {s.mz, s.my, s.mx};
    const int loff[3] = {g.nx * g.ny, g.nx, 1};
    for (int q = 0; q < 3; ++q) {
        if (lower[q] < 0) continue;
        const int l = c - loff[q];
        const RowSlots sl = row_slots(l, g);
        const int up = (q == 0) ? sl.pz : (q == 1) ? sl.py : sl.px;  // block of row l in column c
        double Acl[9], Dl[9], Alc[9], T[9], U[9];
        load9(v + 9 * (base + lower[q]), Acl);
        load9(dinv + 9 * (int64_t)l, Dl);
        load9(v + 9 * ((int64_t)rp[l] + up), Alc);
        mm3(Acl, Dl, T);
        mm3(T, Alc, U);
#pragma unroll
        for (int e = 0; e < 9; ++e) D[e] -= U[e];
    }
    if (!inv3(D, dinv + 9 * (int64_t)c)) atomicCAS(status, 0, (int)RSV_ESINGULAR);
}

__global__ void ilu_fwd_plane(Dims g, const int32_t *__restrict__ rp, const double *__restrict__ v,
                              const int32_t *__restrict__ cells, int p0, int p1, const double *__restrict__ dinv,
                              const double *__restrict__ r, double *y, const int *done) {
    if (done && *(volatile const int *)done) return;
    const int t = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p1) return;
    const int c = cells[t];
    const RowSlots s = row_slots(c, g);
    const int64_t base = rp[c];
    double acc[3] = {r[3 * (int64_t)c], r[3 * (int64_t)c + 1], r[3 * (int64_t)c + 2]};
    const int lower[3] = {s.mz, s.my, s.mx};
    const int loff[3] = {g.nx * g.ny, g.nx, 1};
    for (int q = 0; q < 3; ++q) {
        if (lower[q] < 0) continue;
        const int64_t l = c - loff[q];
        double A[9], xl[3], t3[3];
        load9(v + 9 * (base + lower[q]), A);
        xl[0] = y[3 * l];
        xl[1] = y[3 * l + 1];
        xl[2] = y[3 * l + 2];
        mv3(A, xl, t3);
        acc[0] -= t3[0];
        acc[1] -= t3[1];
        acc[2] -= t3[2];
    }
    double D[9], o[3];
    load9(dinv + 9 * (int64_t)c, D);
    mv3(D, acc, o);
    y[3 * (int64_t)c] = o[0];
    y[3 * (int64_t)c + 1] = o[1];
    y[3 * (int64_t)c + 2] = o[2];
}

__global__ void ilu_bwd_plane(Dims g, const int32_t *__restrict__ rp, const double *__restrict__ v,
                              const int32_t *__restrict__ cells, int p0, int p1, const double *__restrict__ dinv,
                              double *z, const int *done) {
    if (done && *(volatile const int *)done) return;
    const int t = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p1) return;
    const int c = cells[t];
    const RowSlots s = row_slots(c, g);
    const int64_t base = rp[c];
    double acc[3] = {0.0, 0.0, 0.0};
    const int upper[3] = {s.px, s.py, s.pz};
    const int uoff[3] = {1, g.nx, g.nx * g.ny};
    for (int q = 0; q < 3; ++q) {
        if (upper[q] < 0) continue;
        const int64_t u = c + uoff[q];
        double A[9], xu[3], t3[3];
        load9(v + 9 * (base + upper[q]), A);
        xu[0] = z[3 * u];
        xu[1] = z[3 * u + 1];
        xu[2] = z[3 * u + 2];
        mv3(A, xu, t3);
        acc[0] += t3[0];
        acc[1] += t3[1];
        acc[2] += t3[2];
    }
    double D[9], o[3];
    load9(dinv + 9 * (int64_t)c, D);
    mv3(D, acc, o);
    z[3 * (int64_t)c] -= o[0];
    z[3 * (int64_t)c + 1] -= o[1];
    z[3 * (int64_t)c + 2] -= o[2];
}

constexpr int kPlaneThreads = 128;

}  // namespace

cudaError_t build_schedule(const rsv_mat *A, Schedule *sch) {
    const int nx = A->nx, ny = A->ny, nz = A->nz;
    const int nplanes = nx + ny + nz - 2;
    std::vector<int> count(nplanes + 1, 0);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) count[i + j + k + 1]++;
    for (int h = 0; h < nplanes; ++h) count[h + 1] += count[h];
    std::vector<int32_t> cells(A->nb);
    std::vector<int> fill(count.begin(), count.end() - 1);
    for (int64_t c = 0; c < A->nb; ++c) {
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((int64_t)nx * ny));
        cells[fill[i + j + k]++] = (int32_t)c;
    }
    sch->plane_ptr = count;
    sch->nplanes = nplanes;
    cudaError_t e = cudaMallocAsync((void **)&sch->cells, sizeof(int32_t) * std::max<int64_t>(A->nb, 1), A->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(sch->cells, cells.data(), sizeof(int32_t) * A->nb, cudaMemcpyHostToDevice, A->stream);
}

void free_schedule(Schedule *sch) {
    if (sch->cells) cudaFree(sch->cells);
    sch->cells = nullptr;
    sch->plane_ptr.clear();
    sch->nplanes = 0;
}

cudaError_t launch_bj_setup(const rsv_mat *A, double *dinv, int *status) {
    Dims g{A->nx, A->ny, A->nz};
    int grid = (int)((A->nb + 127) / 128);
    rsv::count_launches(1);
    bj_setup_kernel<<<grid, 128, 0, A->stream>>>(A->nb, g, A->d_rp, A->d_v, dinv, status);
    return cudaGetLastError();
}

cudaError_t launch_bj_apply(cudaStream_t st, int64_t nb, const double *dinv, const double *r, double *z,
                            const int *done) {
    int grid = (int)((nb + 127) / 128);
    rsv::count_launches(1);
    bj_apply_kernel<<<grid, 128, 0, st>>>(nb, dinv, r, z, done);
    return cudaGetLastError();
}

cudaError_t launch_ilu_setup(const rsv_mat *A, const Schedule &sch, double *dinv, int *status) {
    Dims g{A->nx, A->ny, A->nz};
    for (int h = 0; h < sch.nplanes; ++h) {
        const int p0 = sch.plane_ptr[h], p1 = sch.plane_ptr[h + 1];
        const int grid = (p1 - p0 + kPlaneThreads - 1) / kPlaneThreads;
        rsv::count_launches(1);
        ilu_factor_plane<<<grid, kPlaneThreads, 0, A->stream>>>(g, A->d_rp, A->d_v, sch.cells, p0, p1, dinv,
                                                                status);
    }
    return cudaGetLastError();
}

cudaError_t launch_ilu_apply(const rsv_mat *A, const Schedule &sch, const double *dinv, const double *r,
                             double *z, const int *done) {
    Dims g{A->nx, A->ny, A->nz};
    for (int h = 0; h < sch.nplanes; ++h) {
        const int p0 = sch.plane_ptr[h], p1 = sch.plane_ptr[h + 1];
        const int grid = (p1 - p0 + kPlaneThreads - 1) / kPlaneThreads;
        rsv::count_launches(1);
        ilu_fwd_plane<<<grid, kPlaneThreads, 0, A->stream>>>(g, A->d_rp, A->d_v, sch.cells, p0, p1, dinv, r, z,
                                                             done);
    }
    for (int h = sch.nplanes - 1; h >= 0; --h) {
        const int p0 = sch.plane_ptr[h], p1 = sch.plane_ptr[h + 1];
        const int grid = (p1 - p0 + kPlaneThreads - 1) / kPlaneThreads;
        rsv::count_launches(1);
        ilu_bwd_plane<<<grid, kPlaneThreads, 0, A->stream>>>(g, A->d_rp, A->d_v, sch.cells, p0, p1, dinv, z,
                                                             done);
    }
    return cudaGetLastError();
}

}  // namespace rsv
