// Block-Jacobi and block ILU(0) preconditioners on the seven-point 3x3-block
// Jacobian.
//
// Block ILU(0) (Section "Restricted Additive Schwarz Method": LU x = b is
// solved as L y = b, U x = y; ILU(0) is the default local solver).  For a
// seven-point pattern the no-fill factor only changes diagonal blocks (the
// grid graph has no triangles), so it is stored as D_c^{-1} with
//     D_c = A_cc - sum_{l in lower(c)} A_cl D_l^{-1} A_lc,
// and applied as M = (D + L_A) D^{-1} (D + U_A) by the tile sweeps of
// ilu_tiles.cu.  Every lower neighbour of cell (i,j,k) lies on hyperplane
// i+j+k-1, so the factorisation runs one launch per hyperplane, all cells of
// a plane in parallel.  This is a legal schedule of the natural-order
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

__device__ __forceinline__ void mm3(const double *a, const double *b, double *c) {
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int f = 0; f < 3; ++f) c[3 * e + f] = a[3 * e] * b[f] + a[3 * e + 1] * b[3 + f] + a[3 * e + 2] * b[6 + f];
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

template <typename Tv>
__device__ __forceinline__ void load9(const Tv *p, double *o) {
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] = (double)p[q];
}

// dinv_c = A_cc^{-1} in FP64 from the FP64 values or their FP32 copy; dinv32
// (optional) receives the FP32 rounding used by mixed-precision applies.
// Grid of global cell c and c's index inside it.
__device__ __forceinline__ Dims grid_of(int64_t c, const SysGrid *sys, const int32_t *sys_of_cell, int &local) {
    const SysGrid g = sys[sys_of_cell[c]];
    local = (int)(c - g.cell0);
    return Dims{g.nx, g.ny, g.nz};
}

template <typename Tv>
__global__ void bj_setup_kernel(int64_t nb, const SysGrid *__restrict__ sys, const int32_t *__restrict__ sys_of_cell,
                                const int32_t *__restrict__ rp, const Tv *__restrict__ v,
                                double *__restrict__ dinv, float *__restrict__ dinv32, int *status) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    int local;
    const Dims g = grid_of(c, sys, sys_of_cell, local);
    const RowSlots s = row_slots(local, g);
    double a[9];
    load9(v + 9 * (int64_t)(rp[c] + s.d), a);
    if (!inv3(a, dinv + 9 * c)) atomicCAS(status, 0, (int)RSV_ESINGULAR);
    if (dinv32)
        for (int q = 0; q < 9; ++q) dinv32[9 * c + q] = (float)dinv[9 * c + q];
}

template <typename T>
__global__ void bj_apply_kernel(int64_t nb, const T *__restrict__ dinv, const T *__restrict__ r, T *__restrict__ z,
                                const int *done) {
    if (done && *(volatile const int *)done) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    T d[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = dinv[9 * c + q];
    const T x0 = r[3 * c], x1 = r[3 * c + 1], x2 = r[3 * c + 2];
    z[3 * c] = d[0] * x0 + d[1] * x1 + d[2] * x2;
    z[3 * c + 1] = d[3] * x0 + d[4] * x1 + d[5] * x2;
    z[3 * c + 2] = d[6] * x0 + d[7] * x1 + d[8] * x2;
}

// D_c = A_cc - sum_{l lower} (A_cl D_l^{-1}) A_lc, lower neighbours in
// ascending column order (-z, -y, -x).
template <typename Tv>
__global__ void ilu_factor_plane(const SysGrid *__restrict__ sys, const int32_t *__restrict__ sys_of_cell,
                                 const int32_t *__restrict__ rp, const Tv *__restrict__ v,
                                 const int32_t *__restrict__ cells, int p0, int p1, double *dinv, int *status) {
    pdl_wait();  // launched with launch_pdl: the previous plane may still be running
    pdl_trigger();
    const int t = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p1) return;
    const int c = cells[t];
    int local;
    const Dims g = grid_of(c, sys, sys_of_cell, local);
    const RowSlots s = row_slots(local, g);
    const int64_t base = rp[c];
    double D[9];
    load9(v + 9 * (base + s.d), D);
    const int lower[3] = {s.mz, s.my, s.mx};
    const int loff[3] = {g.nx * g.ny, g.nx, 1};
    for (int q = 0; q < 3; ++q) {
        if (lower[q] < 0) continue;
        const int l = c - loff[q];
        const RowSlots sl = row_slots(local - loff[q], g);
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

constexpr int kPlaneThreads = 128;

}  // namespace

cudaError_t build_schedule(const rsv_mat *A, Schedule *sch) {
    // hyperplane h = i+j+k inside each grid; plane h of every grid of a batch shares one launch
    int nplanes = 0;
    for (const SysGrid &g : A->h_sys) nplanes = std::max(nplanes, g.nx + g.ny + g.nz - 2);
    std::vector<int> count(nplanes + 1, 0);
    for (const SysGrid &g : A->h_sys)
        for (int k = 0; k < g.nz; ++k)
            for (int j = 0; j < g.ny; ++j)
                for (int i = 0; i < g.nx; ++i) count[i + j + k + 1]++;
    for (int h = 0; h < nplanes; ++h) count[h + 1] += count[h];
    std::vector<int32_t> cells(A->nb);
    std::vector<int> fill(count.begin(), count.end() - 1);
    for (const SysGrid &g : A->h_sys)
        for (int64_t l = 0; l < (int64_t)g.nx * g.ny * g.nz; ++l) {
            const int i = (int)(l % g.nx), j = (int)((l / g.nx) % g.ny), k = (int)(l / ((int64_t)g.nx * g.ny));
            cells[fill[i + j + k]++] = (int32_t)(g.cell0 + l);
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

cudaError_t launch_bj_setup(const rsv_mat *A, bool from_f32, double *dinv, float *dinv32, int *status) {
    int grid = (int)((A->nb + 127) / 128);
    rsv::count_launches(1);
    if (from_f32)
        bj_setup_kernel<float><<<grid, 128, 0, A->stream>>>(A->nb, A->d_sys, A->d_sys_of_cell, A->d_rp, A->d_v32,
                                                            dinv, dinv32, status);
    else
        bj_setup_kernel<double><<<grid, 128, 0, A->stream>>>(A->nb, A->d_sys, A->d_sys_of_cell, A->d_rp, A->d_v,
                                                             dinv, dinv32, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bj_apply(cudaStream_t st, int64_t nb, const T *dinv, const T *r, T *z, const int *done) {
    int grid = (int)((nb + 127) / 128);
    rsv::count_launches(1);
    bj_apply_kernel<T><<<grid, 128, 0, st>>>(nb, dinv, r, z, done);
    return cudaGetLastError();
}
template cudaError_t launch_bj_apply<double>(cudaStream_t, int64_t, const double *, const double *, double *,
                                             const int *);
template cudaError_t launch_bj_apply<float>(cudaStream_t, int64_t, const float *, const float *, float *,
                                            const int *);

// One launch per hyperplane, each a programmatic dependent of the one before (its launch
// overlaps the previous plane; it waits for it on the device before reading its factors).
cudaError_t launch_ilu_setup(const rsv_mat *A, const Schedule &sch, bool from_f32, double *dinv, int *status) {
    for (int h = 0; h < sch.nplanes; ++h) {
        const int p0 = sch.plane_ptr[h], p1 = sch.plane_ptr[h + 1];
        const dim3 grid((p1 - p0 + kPlaneThreads - 1) / kPlaneThreads), block(kPlaneThreads);
        rsv::count_launches(1);
        const cudaError_t e =
            from_f32 ? launch_pdl(ilu_factor_plane<float>, grid, block, 0, A->stream, A->d_sys, A->d_sys_of_cell,
                                  A->d_rp, A->d_v32, sch.cells, p0, p1, dinv, status)
                     : launch_pdl(ilu_factor_plane<double>, grid, block, 0, A->stream, A->d_sys, A->d_sys_of_cell,
                                  A->d_rp, A->d_v, sch.cells, p0, p1, dinv, status);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace rsv
