// Algebraic multigrid for the CPR pressure stage (Section "Algebraic Multigrid
// Methods": the AMG setup algorithm -- strength matrix, a coarse point set that
// is a subset of the fine points, prolongation, R = P^T, Galerkin product
// A_{l+1} = R A_l P, smoothers -- and the V-cycle algorithm).
//
// Setup runs on the host, once per preconditioner setup, on the pressure
// operator the decoupling kernel built on the device (as the paper's AMG
// setup runs on the CPU); the V-cycle runs on the GPU every application.
//   - strength: j != i strongly influences i when -a_ij >= 0.5 max_{k != i}(-a_ik)
//     (the default strength threshold); no strong connections if that maximum <= 0;
//   - coarse points: PMIS.  Measure lambda_i = |{k : i in S_k}| + u_i, u_i the top
//     53 bits of splitmix64(i) as a uniform in [0, 1).  Points nothing depends on
//     (lambda_i < 1) start as F; then in rounds taken from the previous round's
//     state, an undecided point whose measure exceeds every undecided strong
//     neighbour's (S_i and S_i^T) becomes C, and each undecided point that
//     strongly depends on a C point becomes F;
//   - prolongation: identity on C points, direct interpolation on F points,
//     w_ij = -alpha_i a_ij / a_ii over the strong C neighbours j, with
//     alpha_i = (sum of i's off-diagonal entries) / (sum over those neighbours);
//   - smoother: l1-Jacobi, x += D^{-1} (b - A x), D_ii = sum_j |a_ij|, `sweeps`
//     times before and after the coarse correction;
//   - levels while a level has more than max_coarse points (at most max_levels,
//     stopping if a round keeps more than 90% of the points); the coarsest level
//     (at most 1024 points) is solved with its explicit inverse.
// Every level holds its operator, P and R = P^T as CSR (columns ascending), so
// restriction and prolongation are row-parallel products without atomics.
//
// The host setup runs its row loops on all host cores (OpenMP): each CSR is built
// in two passes (row counts, then rows written at their offsets), and every row's
// sums keep their order, so the hierarchy is the same as a one-thread run's.
#include <algorithm>
#include <omp.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace rsv {

struct AmgLevel {
    int n = 0;
    int32_t *rp = nullptr, *ci = nullptr;
    void *v = nullptr, *dl1 = nullptr;           // operator values and l1 row norms (T)
    int32_t *prp = nullptr, *pci = nullptr;      // P: n x n_{l+1}
    void *pv = nullptr;
    int32_t *rrp = nullptr, *rci = nullptr;      // R = P^T: n_{l+1} x n
    void *rv = nullptr;
    void *x = nullptr, *b = nullptr, *r = nullptr;  // T vectors (level 0: x and b are the CPR stage's)
    int64_t nnz = 0;
};

struct Amg {
    int nlev = 0, sweeps = 2, nc = 0;
    bool mixed = false;
    AmgLevel L[kMaxLevels];
    double *minv = nullptr;  // coarsest explicit inverse, FP64 n_c x n_c
    std::vector<void *> allocs;
};

namespace {

struct Csr {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<double> v;
};

double unit_uniform(int64_t i) {
    uint64_t z = (uint64_t)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// rp[i + 1] holds row i's count on entry; on return rp is the row-pointer array.
void prefix_counts(std::vector<int> &rp) {
    for (size_t i = 1; i < rp.size(); ++i) rp[i] += rp[i - 1];
}

// Row i's strong connections (columns ascending), written at out (nullptr: count only).
inline int strong_row(const Csr &A, int i, int *out) {
    double mx = 0.0;
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p)
        if (A.ci[p] != i && -A.v[p] > mx) mx = -A.v[p];
    int m = 0;
    if (mx > 0.0)
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p)
            if (A.ci[p] != i && -A.v[p] >= 0.5 * mx) {
                if (out) out[m] = A.ci[p];
                ++m;
            }
    return m;
}

void strength(const Csr &A, std::vector<int> &srp, std::vector<int> &sci) {
    srp.assign(A.n + 1, 0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A.n; ++i) srp[i + 1] = strong_row(A, i, nullptr);
    prefix_counts(srp);
    sci.assign(srp[A.n], 0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A.n; ++i) strong_row(A, i, sci.data() + srp[i]);
}

// cf: 1 C, -1 F.
void pmis(int n, const std::vector<int> &srp, const std::vector<int> &sci, std::vector<int> &cf) {
    std::vector<int> cnt(n, 0);
    for (int q : sci) cnt[q]++;
    std::vector<int> trp(n + 1, 0), tci(sci.size()), fill(n, 0);
    for (int i = 0; i < n; ++i) trp[i + 1] = trp[i] + cnt[i];
    for (int k = 0; k < n; ++k)
        for (int p = srp[k]; p < srp[k + 1]; ++p) {
            const int i = sci[p];
            tci[trp[i] + fill[i]++] = k;
        }
    std::vector<double> lam(n);
    cf.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        lam[i] = cnt[i] + unit_uniform(i);
        if (lam[i] < 1.0) cf[i] = -1;
    }
    std::vector<char> pick(n), tof(n);
    for (;;) {
        int any = 0;
#pragma omp parallel for schedule(static) reduction(| : any)
        for (int i = 0; i < n; ++i) any |= cf[i] == 0;
        if (!any) break;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
            pick[i] = 0;
            if (cf[i] != 0) continue;
            bool top = true;
            for (int p = srp[i]; p < srp[i + 1] && top; ++p)
                if (cf[sci[p]] == 0 && lam[sci[p]] >= lam[i]) top = false;
            for (int p = trp[i]; p < trp[i + 1] && top; ++p)
                if (cf[tci[p]] == 0 && lam[tci[p]] >= lam[i]) top = false;
            pick[i] = top;
        }
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i)
            if (pick[i]) cf[i] = 1;
        // undecided points that strongly depend on a C point become F (marked first, then set, so
        // every test reads this round's C set only)
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
            tof[i] = 0;
            if (cf[i] != 0) continue;
            for (int p = srp[i]; p < srp[i + 1]; ++p)
                if (cf[sci[p]] == 1) {
                    tof[i] = 1;
                    break;
                }
        }
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i)
            if (tof[i]) cf[i] = -1;
    }
}

// Row i of P (nullptr outputs: count only).
inline int interp_row(const Csr &A, const std::vector<int> &srp, const std::vector<int> &sci,
                      const std::vector<int> &cf, const std::vector<int> &cidx, int i, int *oc, double *ov) {
    if (cf[i] == 1) {
        if (oc) {
            oc[0] = cidx[i];
            ov[0] = 1.0;
        }
        return 1;
    }
    double aii = 0.0, sn = 0.0, sc = 0.0;
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        if (A.ci[p] == i) aii = A.v[p];
        else sn += A.v[p];
    }
    for (int p = srp[i]; p < srp[i + 1]; ++p) {
        const int j = sci[p];
        if (cf[j] != 1) continue;
        for (int r = A.rp[i]; r < A.rp[i + 1]; ++r)
            if (A.ci[r] == j) sc += A.v[r];
    }
    if (!(sc != 0.0 && aii != 0.0)) return 0;
    const double alpha = sn / sc;
    int m = 0;
    for (int p = srp[i]; p < srp[i + 1]; ++p) {
        const int j = sci[p];
        if (cf[j] != 1) continue;
        for (int r = A.rp[i]; r < A.rp[i + 1]; ++r)
            if (A.ci[r] == j) {
                if (oc) {
                    oc[m] = cidx[j];
                    ov[m] = -alpha * A.v[r] / aii;
                }
                ++m;
            }
    }
    return m;
}

void interpolation(const Csr &A, const std::vector<int> &srp, const std::vector<int> &sci, const std::vector<int> &cf,
                   const std::vector<int> &cidx, Csr &P) {
    P.n = A.n;
    P.rp.assign(A.n + 1, 0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A.n; ++i) P.rp[i + 1] = interp_row(A, srp, sci, cf, cidx, i, nullptr, nullptr);
    prefix_counts(P.rp);
    P.ci.assign(P.rp[A.n], 0);
    P.v.assign(P.rp[A.n], 0.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A.n; ++i) interp_row(A, srp, sci, cf, cidx, i, P.ci.data() + P.rp[i], P.v.data() + P.rp[i]);
}

void transpose(const Csr &P, int ncols, Csr &R) {
    R.n = ncols;
    R.rp.assign(ncols + 1, 0);
    for (int q : P.ci) R.rp[q + 1]++;
    for (int I = 0; I < ncols; ++I) R.rp[I + 1] += R.rp[I];
    R.ci.assign(P.ci.size(), 0);
    R.v.assign(P.ci.size(), 0.0);
    std::vector<int> fill(ncols, 0);
    for (int f = 0; f < P.n; ++f)  // rows of R list fine points ascending
        for (int p = P.rp[f]; p < P.rp[f + 1]; ++p) {
            const int I = P.ci[p];
            R.ci[R.rp[I] + fill[I]] = f;
            R.v[R.rp[I] + fill[I]++] = P.v[p];
        }
}

// Ac = R A P: entry (I, J) sums R_If a_fk P_kJ over R's row I (f ascending), A's row f and P's row k, in order.
// The coarse rows are cut into contiguous chunks; each chunk runs with its own dense accumulator and
// writes to its own arrays, and the chunks are then copied into place.
void galerkin(const Csr &A, const Csr &P, const Csr &R, Csr &Ac) {
    const int nc = R.n;
    Ac.n = nc;
    Ac.rp.assign(nc + 1, 0);
    const int nt = std::max(1, std::min(omp_get_max_threads(), nc / 1024 + 1));  // chunks
    std::vector<std::vector<int>> tci(nt);
    std::vector<std::vector<double>> tv(nt);
    std::vector<int> row0(nt + 1);
    for (int t = 0; t <= nt; ++t) row0[t] = (int)((int64_t)nc * t / nt);
#pragma omp parallel for schedule(static, 1)
    for (int t = 0; t < nt; ++t) {
        std::vector<double> acc(nc, 0.0);
        std::vector<int> mark(nc, -1), cols;
        std::vector<int> &oc = tci[t];
        std::vector<double> &ov = tv[t];
        for (int I = row0[t]; I < row0[t + 1]; ++I) {
            cols.clear();
            for (int q = R.rp[I]; q < R.rp[I + 1]; ++q) {
                const int f = R.ci[q];
                const double pf = R.v[q];
                for (int a = A.rp[f]; a < A.rp[f + 1]; ++a) {
                    const int k = A.ci[a];
                    for (int b = P.rp[k]; b < P.rp[k + 1]; ++b) {
                        const int J = P.ci[b];
                        if (mark[J] != I) {
                            mark[J] = I;
                            acc[J] = 0.0;
                            cols.push_back(J);
                        }
                        acc[J] += pf * A.v[a] * P.v[b];
                    }
                }
            }
            std::sort(cols.begin(), cols.end());
            for (int J : cols) {
                oc.push_back(J);
                ov.push_back(acc[J]);
            }
            Ac.rp[I + 1] = (int)cols.size();
        }
    }
    prefix_counts(Ac.rp);
    Ac.ci.assign(Ac.rp[nc], 0);
    Ac.v.assign(Ac.rp[nc], 0.0);
#pragma omp parallel for schedule(static, 1)
    for (int t = 0; t < nt; ++t) {
        std::copy(tci[t].begin(), tci[t].end(), Ac.ci.begin() + Ac.rp[row0[t]]);
        std::copy(tv[t].begin(), tv[t].end(), Ac.v.begin() + Ac.rp[row0[t]]);
    }
}

template <typename T>
__global__ void amg_jacobi_first(int n, const T *__restrict__ dl1, const T *__restrict__ b, T *__restrict__ x,
                                 const int *done) {
    if (done && *(volatile const int *)done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = T(0) + b[i] / dl1[i];
}

// r = b - A x
template <typename T>
__global__ void amg_residual(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const T *__restrict__ v, const T *__restrict__ b, const T *__restrict__ x,
                             T *__restrict__ r, const int *done) {
    if (done && *(volatile const int *)done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T s = T(0);
    for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * x[ci[p]];
    r[i] = b[i] - s;
}

template <typename T>
__global__ void amg_jacobi_update(int n, const T *__restrict__ dl1, const T *__restrict__ r, T *__restrict__ x,
                                  const int *done) {
    if (done && *(volatile const int *)done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += r[i] / dl1[i];
}

// y = M u (assign) or y += M u, M in CSR.
template <typename T, bool ADD>
__global__ void amg_csr_apply(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const T *__restrict__ v, const T *__restrict__ u, T *__restrict__ y, const int *done) {
    if (done && *(volatile const int *)done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T s = T(0);
    for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * u[ci[p]];
    y[i] = ADD ? y[i] + s : s;
}

// x = Minv b, one warp per row, FP64 arithmetic.
template <typename T>
__global__ void amg_coarse_apply(int n, const double *__restrict__ Minv, const T *__restrict__ b, T *__restrict__ x,
                                 const int *done) {
    if (done && *(volatile const int *)done) return;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int q = lane; q < n; q += 32) s += Minv[(int64_t)row * n + q] * (double)b[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = (T)s;
}

unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// Gauss-Jordan inverse with partial pivoting on the host (n <= 1024), for the coarsest level.
bool dense_inverse(int n, std::vector<double> M, std::vector<double> &inv) {
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(M[(size_t)i * n + k]) > std::fabs(M[(size_t)p * n + k])) p = i;
        if (!(std::fabs(M[(size_t)p * n + k]) > 1e-300)) return false;
        if (p != k)
            for (int q = 0; q < n; ++q) {
                std::swap(M[(size_t)k * n + q], M[(size_t)p * n + q]);
                std::swap(inv[(size_t)k * n + q], inv[(size_t)p * n + q]);
            }
        const double d = M[(size_t)k * n + k];
        for (int q = 0; q < n; ++q) {
            M[(size_t)k * n + q] /= d;
            inv[(size_t)k * n + q] /= d;
        }
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            const double f = M[(size_t)i * n + k];
            if (f == 0.0) continue;
            for (int q = 0; q < n; ++q) {
                M[(size_t)i * n + q] -= f * M[(size_t)k * n + q];
                inv[(size_t)i * n + q] -= f * inv[(size_t)k * n + q];
            }
        }
    }
    return true;
}

}  // namespace

void amg_free(Cpr *P) {
    Amg *g = (Amg *)P->amg;
    if (!g) return;
    for (void *p : g->allocs) cudaFree(p);
    delete g;
    P->amg = nullptr;
}

rsv_status amg_info(const Cpr &P, int *nlev, int64_t *sizes) {
    const Amg *g = (const Amg *)P.amg;
    if (!g) return RSV_EINVAL;
    if (nlev) *nlev = g->nlev;
    if (sizes)
        for (int l = 0; l < g->nlev; ++l) {
            sizes[2 * l] = g->L[l].n;
            sizes[2 * l + 1] = g->L[l].nnz;
        }
    return RSV_OK;
}

// Build the algebraic hierarchy from the finest pressure stencil P->a7[0] (FP64, slot-major
// [7][nb] on the device; slots -z, -y, -x, centre, +x, +y, +z).  Level 0's vectors are the
// CPR stage's P->x[0] / P->b[0].
rsv_status amg_setup(const rsv_mat *A, Cpr *P, int max_levels, int max_coarse, int sweeps) {
    amg_free(P);
    const int nx = A->nx, ny = A->ny, nz = A->nz;
    const int64_t nb = A->nb;
    cudaStream_t st = A->stream;
    std::vector<double> a7((size_t)7 * nb);
    RSV_CUDA_TRY(cudaMemcpyAsync(a7.data(), P->a7[0], sizeof(double) * 7 * nb, cudaMemcpyDeviceToHost, st));
    RSV_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<Csr> As(1), Ps, Rs;
    {
        // the pressure operator has the matrix's own seven-point pattern (slots -z, -y, -x, self, +x,
        // +y, +z; absent faces skipped): take its row pointers and columns, fill the values per row
        Csr &A0 = As[0];
        A0.n = (int)nb;
        A0.rp.assign(A->h_rp.begin(), A->h_rp.end());
        A0.ci.assign(A->h_ci.begin(), A->h_ci.end());
        A0.v.assign(A0.ci.size(), 0.0);
        static const int DI[7] = {0, 0, -1, 0, 1, 0, 0}, DJ[7] = {0, -1, 0, 0, 0, 1, 0}, DK[7] = {-1, 0, 0, 0, 0, 0, 1};
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < nb; ++c) {
            const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((int64_t)nx * ny));
            int p = A0.rp[c];
            for (int s = 0; s < 7; ++s) {
                const int ii = i + DI[s], jj = j + DJ[s], kk = k + DK[s];
                if (ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz) continue;
                A0.v[p++] = a7[(size_t)s * nb + c];
            }
        }
    }
    max_levels = std::min(std::max(max_levels, 1), kMaxLevels);
    while ((int)As.size() < max_levels && As.back().n > max_coarse) {
        const Csr &Al = As.back();
        std::vector<int> srp, sci, cf, cidx(Al.n, -1);
        strength(Al, srp, sci);
        pmis(Al.n, srp, sci, cf);
        int nc = 0;
        for (int i = 0; i < Al.n; ++i)
            if (cf[i] == 1) cidx[i] = nc++;
        if (nc == 0 || nc > 0.9 * Al.n) break;
        Csr Pl, Rl, Ac;
        interpolation(Al, srp, sci, cf, cidx, Pl);
        transpose(Pl, nc, Rl);
        galerkin(Al, Pl, Rl, Ac);
        Ps.push_back(std::move(Pl));
        Rs.push_back(std::move(Rl));
        As.push_back(std::move(Ac));
    }
    const int nlev = (int)As.size();
    const int nc = As.back().n;
    if (nc > 1024) return RSV_ENOTSUP;  // the coarsest level must be small enough for its explicit inverse
    std::vector<double> dense((size_t)nc * nc, 0.0), inv;
    for (int i = 0; i < nc; ++i)
        for (int p = As.back().rp[i]; p < As.back().rp[i + 1]; ++p) dense[(size_t)i * nc + As.back().ci[p]] += As.back().v[p];
    if (!dense_inverse(nc, dense, inv)) return RSV_ESINGULAR;

    Amg *g = new (std::nothrow) Amg();
    if (!g) return RSV_ENOMEM;
    P->amg = g;
    g->nlev = nlev;
    g->sweeps = sweeps;
    g->mixed = P->mixed;
    g->nc = nc;
    const size_t es = P->mixed ? sizeof(float) : sizeof(double);
    cudaError_t e = cudaSuccess;
    auto dalloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) g->allocs.push_back(p);
        return p;
    };
    auto up_i = [&](const std::vector<int> &h) -> int32_t * {
        int32_t *d = (int32_t *)dalloc(sizeof(int32_t) * h.size());
        if (e == cudaSuccess && !h.empty()) e = cudaMemcpyAsync(d, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, st);
        return d;
    };
    std::vector<std::vector<float>> keep32;
    auto up_v = [&](const std::vector<double> &h) -> void * {
        void *d = dalloc(es * h.size());
        if (e != cudaSuccess || h.empty()) return d;
        if (!P->mixed) {
            e = cudaMemcpyAsync(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st);
        } else {
            keep32.emplace_back(h.begin(), h.end());  // rounded to float
            e = cudaMemcpyAsync(d, keep32.back().data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st);
        }
        return d;
    };
    for (int l = 0; l < nlev; ++l) {
        AmgLevel &L = g->L[l];
        const Csr &Al = As[l];
        L.n = Al.n;
        L.nnz = (int64_t)Al.ci.size();
        L.rp = up_i(Al.rp);
        L.ci = up_i(Al.ci);
        L.v = up_v(Al.v);
        std::vector<double> d(Al.n, 0.0);
        for (int i = 0; i < Al.n; ++i) {
            double s = 0.0;
            for (int p = Al.rp[i]; p < Al.rp[i + 1]; ++p) s += std::fabs(Al.v[p]);
            d[i] = s;
        }
        L.dl1 = up_v(d);
        if (l + 1 < nlev) {
            L.prp = up_i(Ps[l].rp);
            L.pci = up_i(Ps[l].ci);
            L.pv = up_v(Ps[l].v);
            L.rrp = up_i(Rs[l].rp);
            L.rci = up_i(Rs[l].ci);
            L.rv = up_v(Rs[l].v);
        }
        if (l == 0) {
            L.x = P->x[0];
            L.b = P->b[0];
        } else {
            L.x = dalloc(es * Al.n);
            L.b = dalloc(es * Al.n);
        }
        L.r = dalloc(es * Al.n);
    }
    g->minv = (double *)dalloc(sizeof(double) * inv.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->minv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host staging buffers go out of scope
    if (e != cudaSuccess) {
        amg_free(P);
        return cuda_status(e);
    }
    return RSV_OK;
}

template <typename T>
static cudaError_t amg_cycle(const Amg &g, int l, cudaStream_t st, const int *done) {
    const AmgLevel &L = g.L[l];
    T *x = (T *)L.x, *b = (T *)L.b, *r = (T *)L.r;
    const T *v = (const T *)L.v, *dl1 = (const T *)L.dl1;
    const unsigned bl = nblk(L.n);
    if (l == g.nlev - 1) {
        count_launches(1);
        amg_coarse_apply<T><<<nblk((int64_t)L.n * 32), 256, 0, st>>>(L.n, g.minv, b, x, done);
        return cudaGetLastError();
    }
    // pre-smoothing from x = 0 (the first sweep is x = D^{-1} b)
    if (g.sweeps == 0) {
        count_launches(1);
        cudaError_t e = cudaMemsetAsync(x, 0, sizeof(T) * L.n, st);
        if (e != cudaSuccess) return e;
    }
    for (int s = 0; s < g.sweeps; ++s) {
        if (s == 0) {
            count_launches(1);
            amg_jacobi_first<T><<<bl, 256, 0, st>>>(L.n, dl1, b, x, done);
        } else {
            count_launches(2);
            amg_residual<T><<<bl, 256, 0, st>>>(L.n, L.rp, L.ci, v, b, x, r, done);
            amg_jacobi_update<T><<<bl, 256, 0, st>>>(L.n, dl1, r, x, done);
        }
    }
    const AmgLevel &C = g.L[l + 1];
    count_launches(2);
    amg_residual<T><<<bl, 256, 0, st>>>(L.n, L.rp, L.ci, v, b, x, r, done);
    amg_csr_apply<T, false><<<nblk(C.n), 256, 0, st>>>(C.n, L.rrp, L.rci, (const T *)L.rv, r, (T *)C.b, done);
    cudaError_t e = amg_cycle<T>(g, l + 1, st, done);
    if (e != cudaSuccess) return e;
    count_launches(1);
    amg_csr_apply<T, true><<<bl, 256, 0, st>>>(L.n, L.prp, L.pci, (const T *)L.pv, (const T *)C.x, x, done);
    for (int s = 0; s < g.sweeps; ++s) {
        count_launches(2);
        amg_residual<T><<<bl, 256, 0, st>>>(L.n, L.rp, L.ci, v, b, x, r, done);
        amg_jacobi_update<T><<<bl, 256, 0, st>>>(L.n, dl1, r, x, done);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t amg_vcycle(const Cpr &P, cudaStream_t st, const int *done) {
    const Amg *g = (const Amg *)P.amg;
    if (!g) return cudaErrorInvalidValue;
    return amg_cycle<T>(*g, 0, st, done);
}

template cudaError_t amg_vcycle<double>(const Cpr &, cudaStream_t, const int *);
template cudaError_t amg_vcycle<float>(const Cpr &, cudaStream_t, const int *);

}  // namespace rsv
