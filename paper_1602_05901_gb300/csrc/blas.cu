// Vector algebra of the Krylov solvers (Section "Algebraic Operations":
// y = a x + b y, <x,y>, ||x||), fused where a solver step allows it.
//
// Vectors are FP64, or FP32 in the inner solves of mixed precision.  Every
// reduction is far more accurate than its vectors: FP64 vectors accumulate with
// FP64 FMAs (FP64-accurate sums); FP32
// vectors accumulate each thread's products in double-float form (an FP32
// pair hi + lo updated with error-free transformations: the exact rounding
// error of each product from an FMA, and of each addition from Knuth's
// two-sum), which GB300 runs on its FP32 pipes instead of its much narrower
// FP64 pipe.  The warp trees add those pairs as double-float sums too; one
// value per warp is widened to FP64 for the block and grid reductions.  An FP32
// vector's sums so keep about 46 bits, against the 24 of its entries.
//
// Reductions are deterministic: every CTA writes one partial per output, and
// the last CTA to finish (ticket counter) sums the partials in CTA order.
// Rows are processed as 16-byte vectors when every pointer and the basis
// leading dimension allow it.
#include "reduce.cuh"

namespace rsv {
namespace {

constexpr int kGroup = 16;  // basis vectors reduced per pass in the multi-dot

__device__ __forceinline__ bool is_done(const int *done) { return done && *(volatile const int *)done; }

// Returns true in exactly one CTA: the last one to pass, after every CTA's
// partials are visible.
__device__ __forceinline__ bool last_cta(unsigned *counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    return am_last;
}

// Block-reduce one partial sum per thread into partial[slot * grid + block]: a warp
// tree in the accumulator's form, then the warps' sums in FP64 in warp order.
template <typename T>
__device__ __forceinline__ void block_partial(Part<T> v, double *sm, double *partial, int slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v.add(v.xor_shfl(o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v.value();
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) s += sm[q];
        partial[(int64_t)slot * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
}

// Block-reduce kGroup partial sums per thread (the first kg are kept) into
// partial[(slot0 + i) * grid + block].  The warp stage is a butterfly: at each of
// the first four levels a lane keeps half of its values, sends the other half to
// its partner and adds what it receives, so a lane ends with one value, the sum
// over 16 lanes of value (lane >> 1); the fifth level adds the partner's.  That is
// 16 exchanges and additions per lane instead of 5 per value.  Then the warps'
// sums are added in FP64 in warp order (fixed order: deterministic).
template <typename T>
__device__ __forceinline__ void block_partial_group(Part<T> (&v)[kGroup], int kg, double (*sm)[kRedThreads / 32],
                                                    double *partial, int slot0) {
    static_assert(kGroup == 16, "the butterfly halves 16 values four times");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const bool up = (lane & (2 * h)) != 0;  // this lane keeps the upper half
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const Part<T> send = up ? v[i] : v[i + h];
            Part<T> keep = up ? v[i + h] : v[i];
            keep.add(send.xor_shfl(2 * h));
            v[i] = keep;
        }
    }
    v[0].add(v[0].xor_shfl(1));
    if ((lane & 1) == 0 && (lane >> 1) < kg) sm[lane >> 1][warp] = v[0].value();
    __syncthreads();
    if (threadIdx.x < kg) {
        double s = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) s += sm[threadIdx.x][q];
        partial[(int64_t)(slot0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
}

// out[i] = <w, V_i> for i < k; if self_nrm, also out[k] = <w, w> and *self_nrm = ||w||.
// Final reduction in the last CTA: warp w sums the gridDim.x partials of
// outputs w, w + 8, ...; each lane adds a fixed strided subset, then a
// shuffle tree combines the lanes (a fixed order: deterministic).
__device__ __forceinline__ double final_sum(const double *partial, int slot) {
    double s = 0.0;
    for (unsigned b = threadIdx.x & 31; b < gridDim.x; b += 32) s += __ldcg(&partial[(int64_t)slot * gridDim.x + b]);
    return warp_sum(s);
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads, 2) mdot_kernel(int64_t n, const T *__restrict__ w,
                                                           const T *__restrict__ V, int64_t ldv, int k,
                                                           double *partial, double *out, double *self_nrm,
                                                           unsigned *counter, const int *done, const int *skip) {
    if (is_done(done) || is_done(skip)) return;
    using VT = Vec<T>;
    __shared__ double sm[kRedThreads / 32];
    __shared__ double smg[kGroup][kRedThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // <w, w> rides along with the first group of projections (w is read once); alone only when k == 0
    const bool fold = self_nrm && k > 0;
    Acc<T> ww;
    if (self_nrm && !fold) {
        Acc<T> &a = ww;
        if (VEC) {
            const int64_t nv = n / VT::N;
            for (int64_t r = tid; r < nv; r += stride) {
                const typename VT::V wr = reinterpret_cast<const typename VT::V *>(w)[r];
#pragma unroll
                for (int q = 0; q < VT::N; ++q) a.add(VT::get(wr, q), VT::get(wr, q));
            }
            for (int64_t r = nv * VT::N + tid; r < n; r += stride) a.add(w[r], w[r]);
        } else {
            for (int64_t r = tid; r < n; r += stride) a.add(w[r], w[r]);
        }
    }
    for (int g0 = 0; g0 < k; g0 += kGroup) {
        Acc<T> acc[kGroup];
        const int kg = min(kGroup, k - g0);
        if (VEC) {
            const int64_t nv = n / VT::N;
            const bool nw = fold && g0 == 0;
            for (int64_t r = tid; r < nv; r += stride) {
                // issue every load of the group first, then accumulate (keeps kg loads in flight)
                const typename VT::V wr = reinterpret_cast<const typename VT::V *>(w)[r];
                typename VT::V vr[kGroup];
#pragma unroll
                for (int i = 0; i < kGroup; ++i)
                    if (i < kg) vr[i] = reinterpret_cast<const typename VT::V *>(V + (int64_t)(g0 + i) * ldv)[r];
                if (nw) {
#pragma unroll
                    for (int q = 0; q < VT::N; ++q) ww.add(VT::get(wr, q), VT::get(wr, q));
                }
#pragma unroll
                for (int i = 0; i < kGroup; ++i)
                    if (i < kg) {
#pragma unroll
                        for (int q = 0; q < VT::N; ++q) acc[i].add(VT::get(wr, q), VT::get(vr[i], q));
                    }
            }
            for (int64_t r = nv * VT::N + tid; r < n; r += stride) {
                if (nw) ww.add(w[r], w[r]);
#pragma unroll
                for (int i = 0; i < kGroup; ++i)
                    if (i < kg) acc[i].add(w[r], V[(int64_t)(g0 + i) * ldv + r]);
            }
        } else {
            const bool nw = fold && g0 == 0;
            for (int64_t r = tid; r < n; r += stride) {
                const T wr = w[r];
                if (nw) ww.add(wr, wr);
#pragma unroll
                for (int i = 0; i < kGroup; ++i)
                    if (i < kg) acc[i].add(wr, V[(int64_t)(g0 + i) * ldv + r]);
            }
        }
        Part<T> vals[kGroup];
#pragma unroll
        for (int i = 0; i < kGroup; ++i) vals[i] = i < kg ? Part<T>::of(acc[i]) : Part<T>::zero();
        block_partial_group<T>(vals, kg, smg, partial, g0);
    }
    if (self_nrm) block_partial<T>(Part<T>::of(ww), sm, partial, k);
    if (last_cta(counter)) {
        const int kk = self_nrm ? k + 1 : k;
        for (int i = threadIdx.x >> 5; i < kk; i += kRedThreads / 32) {
            const double s = final_sum(partial, i);
            if ((threadIdx.x & 31) == 0) {
                out[i] = s;
                if (i == k) *self_nrm = sqrt(s);
            }
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// Two multi-vector dot products in one read of the basis: ow[i] = <w, V_i> and
// ou[i] = <u, V_i> for i < k (u is typically a column of V itself).  Groups of
// eight basis vectors per pass over w and u, so a group's sixteen sums go
// through the same butterfly reduction as the one-vector multi-dot.  Partial
// slots: 2 g0 + i (w) and 2 g0 + 8 + i (u) for the group starting at g0.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads, 2) mdot2_kernel(int64_t n, const T *__restrict__ w,
                                                            const T *__restrict__ u, const T *__restrict__ V,
                                                            int64_t ldv, int k, double *partial, double *ow,
                                                            double *ou, unsigned *counter, const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (is_done(done)) return;
    using VT = Vec<T>;
    constexpr int G2 = kGroup / 2;
    __shared__ double smg[kGroup][kRedThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int g0 = 0; g0 < k; g0 += G2) {
        Acc<T> aw[G2], au[G2];
        const int kg = min(G2, k - g0);
        int64_t tail = 0;
        if (VEC) {
            const int64_t nv = n / VT::N;
            for (int64_t r = tid; r < nv; r += stride) {
                const typename VT::V wr = reinterpret_cast<const typename VT::V *>(w)[r];
                const typename VT::V ur = reinterpret_cast<const typename VT::V *>(u)[r];
                typename VT::V vr[G2];
#pragma unroll
                for (int i = 0; i < G2; ++i)
                    if (i < kg) vr[i] = reinterpret_cast<const typename VT::V *>(V + (int64_t)(g0 + i) * ldv)[r];
#pragma unroll
                for (int i = 0; i < G2; ++i)
                    if (i < kg) {
#pragma unroll
                        for (int q = 0; q < VT::N; ++q) {
                            aw[i].add(VT::get(wr, q), VT::get(vr[i], q));
                            au[i].add(VT::get(ur, q), VT::get(vr[i], q));
                        }
                    }
            }
            tail = nv * VT::N;
        }
        for (int64_t r = tail + tid; r < n; r += stride) {
            const T wr = w[r], ur = u[r];
#pragma unroll
            for (int i = 0; i < G2; ++i)
                if (i < kg) {
                    const T vv = V[(int64_t)(g0 + i) * ldv + r];
                    aw[i].add(wr, vv);
                    au[i].add(ur, vv);
                }
        }
        Part<T> vals[kGroup];
#pragma unroll
        for (int i = 0; i < G2; ++i) {
            vals[i] = i < kg ? Part<T>::of(aw[i]) : Part<T>::zero();
            vals[G2 + i] = i < kg ? Part<T>::of(au[i]) : Part<T>::zero();
        }
        block_partial_group<T>(vals, kGroup, smg, partial, 2 * g0);
    }
    if (last_cta(counter)) {
        for (int i = threadIdx.x >> 5; i < 2 * k; i += kRedThreads / 32) {
            const int vec = i / k, q = i - vec * k;  // output vec (0: w, 1: u), basis index q
            const int slot = 2 * (q / G2) * G2 + vec * G2 + q % G2;
            const double sum = final_sum(partial, slot);
            if ((threadIdx.x & 31) == 0) (vec ? ou : ow)[q] = sum;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// out = base + sgn * sum_i c_i V_i, in the vector precision; ||out|| summed like the dot products.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads) maxpy_kernel(int64_t n, const T *base, const T *__restrict__ V,
                                                            int64_t ldv, int k, const double *c, double sgn, T *out,
                                                            double *partial, double *nrm, unsigned *counter,
                                                            const int *done, const int *skip) {
    if (is_done(done) || is_done(skip)) return;
    using VT = Vec<T>;
    __shared__ T sc[kMaxRestart + 1];
    __shared__ double sm[kRedThreads / 32];
    for (int i = threadIdx.x; i < k; i += blockDim.x) sc[i] = (T)(sgn * c[i]);
    __syncthreads();
    Acc<T> ss;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tail = 0;
    if (VEC) {
        const int64_t nv = n / VT::N;
        for (int64_t r = tid; r < nv; r += stride) {
            typename VT::V acc;
            if (base)
                acc = reinterpret_cast<const typename VT::V *>(base)[r];
            else
                for (int q = 0; q < VT::N; ++q) VT::set(acc, q, T(0));
            constexpr int B = 8;  // loads issued together
            for (int i0 = 0; i0 < k; i0 += B) {
                typename VT::V vr[B];
#pragma unroll
                for (int i = 0; i < B; ++i)
                    if (i0 + i < k) vr[i] = reinterpret_cast<const typename VT::V *>(V + (int64_t)(i0 + i) * ldv)[r];
#pragma unroll
                for (int i = 0; i < B; ++i)
                    if (i0 + i < k) {
#pragma unroll
                        for (int q = 0; q < VT::N; ++q)
                            VT::set(acc, q, fma(sc[i0 + i], VT::get(vr[i], q), VT::get(acc, q)));
                    }
            }
            reinterpret_cast<typename VT::V *>(out)[r] = acc;
#pragma unroll
            for (int q = 0; q < VT::N; ++q) ss.add(VT::get(acc, q), VT::get(acc, q));
        }
        tail = nv * VT::N;
    }
    for (int64_t r = tail + tid; r < n; r += stride) {
        T acc = base ? base[r] : T(0);
        for (int i = 0; i < k; ++i) acc = fma(sc[i], V[(int64_t)i * ldv + r], acc);
        out[r] = acc;
        ss.add(acc, acc);
    }
    if (!nrm) return;
    block_partial<T>(Part<T>::of(ss), sm, partial, 0);
    if (last_cta(counter)) {
        if (threadIdx.x < 32) {
            const double s = final_sum(partial, 0);
            if (threadIdx.x == 0) {
                *nrm = sqrt(s);
                *counter = 0u;
            }
        }
    }
}

// Classical Gram-Schmidt with reorthogonalisation, the first pass's update fused with the
// second pass's projections (Section "Algebraic Operations": the orthogonalisation of
// GMRES is dot products and vector updates).  For each row block a thread loads the k
// basis values once into registers, forms w' = w - sum_i c_i V_i with the same FMA order
// as maxpy_kernel, stores it, and accumulates <w', V_i> and <w', w'> from those registers:
// the second pass's projections cost no second read of the basis.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads, 1) maxpy_mdot_kernel(int64_t n, T *w, const T *__restrict__ V,
                                                                 int64_t ldv, int k, const double *c,
                                                                 double *partial, double *proj, double *nrm,
                                                                 unsigned *counter, const int *done) {
    if (is_done(done)) return;
    using VT = Vec<T>;
    constexpr int KF = kFuseMax<T>;
    __shared__ T sc[KF];
    __shared__ double smg[kGroup][kRedThreads / 32];
    for (int i = threadIdx.x; i < k; i += blockDim.x) sc[i] = (T)(-c[i]);
    __syncthreads();
    Acc<T> ss, acc[KF];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tail = 0;
    if (VEC) {
        const int64_t nv = n / VT::N;
        for (int64_t r = tid; r < nv; r += stride) {
            typename VT::V vr[KF];
#pragma unroll
            for (int i = 0; i < KF; ++i)
                if (i < k) vr[i] = reinterpret_cast<const typename VT::V *>(V + (int64_t)i * ldv)[r];
            typename VT::V o = reinterpret_cast<const typename VT::V *>(w)[r];
#pragma unroll
            for (int i = 0; i < KF; ++i)
                if (i < k) {
#pragma unroll
                    for (int q = 0; q < VT::N; ++q) VT::set(o, q, fma(sc[i], VT::get(vr[i], q), VT::get(o, q)));
                }
            reinterpret_cast<typename VT::V *>(w)[r] = o;
#pragma unroll
            for (int q = 0; q < VT::N; ++q) ss.add(VT::get(o, q), VT::get(o, q));
#pragma unroll
            for (int i = 0; i < KF; ++i)
                if (i < k) {
#pragma unroll
                    for (int q = 0; q < VT::N; ++q) acc[i].add(VT::get(o, q), VT::get(vr[i], q));
                }
        }
        tail = nv * VT::N;
    }
    for (int64_t r = tail + tid; r < n; r += stride) {
        T vr[KF];
#pragma unroll
        for (int i = 0; i < KF; ++i)
            if (i < k) vr[i] = V[(int64_t)i * ldv + r];
        T o = w[r];
#pragma unroll
        for (int i = 0; i < KF; ++i)
            if (i < k) o = fma(sc[i], vr[i], o);
        w[r] = o;
        ss.add(o, o);
#pragma unroll
        for (int i = 0; i < KF; ++i)
            if (i < k) acc[i].add(o, vr[i]);
    }
#pragma unroll
    for (int g0 = 0; g0 < KF; g0 += kGroup) {
        if (g0 < k) {
            Part<T> vals[kGroup];
#pragma unroll
            for (int i = 0; i < kGroup; ++i) vals[i] = g0 + i < k ? Part<T>::of(acc[g0 + i]) : Part<T>::zero();
            block_partial_group<T>(vals, min(kGroup, k - g0), smg, partial, g0);
        }
    }
    block_partial<T>(Part<T>::of(ss), &smg[0][0], partial, k);
    if (last_cta(counter)) {
        for (int i = threadIdx.x >> 5; i <= k; i += kRedThreads / 32) {
            const double s = final_sum(partial, i);
            if ((threadIdx.x & 31) == 0) {
                if (i < k)
                    proj[i] = s;
                else
                    *nrm = sqrt(s);
            }
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// The update pass of a delayed CGS2 step (GMRES): from one read of V_0..V_{k-1}, u and w,
//   u <- cS[0] u - sum_i cB[i] V_i                    (the reorthogonalised, normalised v_k)
//   w <- cS[0] w - cS[1] u_old - sum_i cA[i] V_i      (the next step's once-orthogonalised vector)
// Both outputs are written over their inputs by the thread that read them.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads) dcgs2_update_kernel(int64_t n, T *u, T *w, const T *__restrict__ V,
                                                                   int64_t ldv, int k, const double *cA,
                                                                   const double *cB, const double *cS,
                                                                   const int *done) {
    pdl_wait();  // launched with launch_pdl: the previous kernel may still be running
    pdl_trigger();
    if (is_done(done)) return;
    using VT = Vec<T>;
    __shared__ T sa[kMaxRestart], sb[kMaxRestart];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        sa[i] = (T)(-cA[i]);
        sb[i] = (T)(-cB[i]);
    }
    __syncthreads();
    const T cw = (T)cS[0], cu = (T)(-cS[1]);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tail = 0;
    if (VEC) {
        const int64_t nv = n / VT::N;
        for (int64_t r = tid; r < nv; r += stride) {
            const typename VT::V ur = reinterpret_cast<const typename VT::V *>(u)[r];
            const typename VT::V wr = reinterpret_cast<const typename VT::V *>(w)[r];
            typename VT::V av, aw;
#pragma unroll
            for (int q = 0; q < VT::N; ++q) {
                VT::set(av, q, VT::get(ur, q) * cw);
                VT::set(aw, q, fma(cu, VT::get(ur, q), VT::get(wr, q) * cw));
            }
            constexpr int B = 8;  // loads issued together
            for (int i0 = 0; i0 < k; i0 += B) {
                typename VT::V vr[B];
#pragma unroll
                for (int i = 0; i < B; ++i)
                    if (i0 + i < k) vr[i] = reinterpret_cast<const typename VT::V *>(V + (int64_t)(i0 + i) * ldv)[r];
#pragma unroll
                for (int i = 0; i < B; ++i)
                    if (i0 + i < k) {
#pragma unroll
                        for (int q = 0; q < VT::N; ++q) {
                            VT::set(av, q, fma(sb[i0 + i], VT::get(vr[i], q), VT::get(av, q)));
                            VT::set(aw, q, fma(sa[i0 + i], VT::get(vr[i], q), VT::get(aw, q)));
                        }
                    }
            }
            reinterpret_cast<typename VT::V *>(u)[r] = av;
            reinterpret_cast<typename VT::V *>(w)[r] = aw;
        }
        tail = nv * VT::N;
    }
    for (int64_t r = tail + tid; r < n; r += stride) {
        const T ur = u[r];
        T av = ur * cw, aw = fma(cu, ur, w[r] * cw);
        for (int i = 0; i < k; ++i) {
            const T v = V[(int64_t)i * ldv + r];
            av = fma(sb[i], v, av);
            aw = fma(sa[i], v, aw);
        }
        u[r] = av;
        w[r] = aw;
    }
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads) dot_kernel(int64_t n, const T *__restrict__ x,
                                                          const T *__restrict__ y, double *partial, double *out,
                                                          unsigned *counter, int sqrt_out, const int *done) {
    if (is_done(done)) return;
    using VT = Vec<T>;
    __shared__ double sm[kRedThreads / 32];
    Acc<T> acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tail = 0;
    if (VEC) {
        const int64_t nv = n / VT::N;
        for (int64_t r = tid; r < nv; r += stride) {
            const typename VT::V a = reinterpret_cast<const typename VT::V *>(x)[r];
            const typename VT::V b = reinterpret_cast<const typename VT::V *>(y)[r];
#pragma unroll
            for (int q = 0; q < VT::N; ++q) acc.add(VT::get(a, q), VT::get(b, q));
        }
        tail = nv * VT::N;
    }
    for (int64_t r = tail + tid; r < n; r += stride) acc.add(x[r], y[r]);
    block_partial<T>(Part<T>::of(acc), sm, partial, 0);
    if (last_cta(counter)) {
        if (threadIdx.x < 32) {
            const double s = final_sum(partial, 0);
            if (threadIdx.x == 0) {
                *out = sqrt_out ? sqrt(s) : s;
                *counter = 0u;
            }
        }
    }
}

template <typename T>
__global__ void axpby_kernel(int64_t n, T a, const T *x, T b, const T *y, T *z) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride)
        z[r] = (b == T(0)) ? a * x[r] : a * x[r] + b * y[r];
}

// The FP64 reciprocal of a device scalar, formed once per block (an FP64 division in
// every thread costs more than the whole vector pass on GB300's narrow FP64 pipe).
__device__ __forceinline__ double block_inverse(const double *s) {
    __shared__ double f;
    if (threadIdx.x == 0) f = 1.0 / *s;
    __syncthreads();
    return f;
}

template <typename T, bool VEC>
__global__ void scale_inv_kernel(int64_t n, T *x, const double *s, const int *done) {
    if (is_done(done)) return;
    using VT = Vec<T>;
    const T f = (T)block_inverse(s);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tail = 0;
    if (VEC) {
        const int64_t nv = n / VT::N;
        for (int64_t r = tid; r < nv; r += stride) {
            typename VT::V v = reinterpret_cast<typename VT::V *>(x)[r];
#pragma unroll
            for (int q = 0; q < VT::N; ++q) VT::set(v, q, VT::get(v, q) * f);
            reinterpret_cast<typename VT::V *>(x)[r] = v;
        }
        tail = nv * VT::N;
    }
    for (int64_t r = tail + tid; r < n; r += stride) x[r] *= f;
}

// Mixed-precision glue: xf = (float)(x / *s); x += (*s) * (double)df.
__global__ void to_f32_scaled(int64_t n, const double *__restrict__ x, const double *s, float *__restrict__ xf) {
    const double f = block_inverse(s);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) xf[r] = (float)(x[r] * f);
}

__global__ void add_f32_scaled(int64_t n, const float *__restrict__ df, const double *s, double *__restrict__ x) {
    const double f = *s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) x[r] += f * (double)df[r];
}

int elementwise_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T>
bool vec_ok(int64_t ldv, std::initializer_list<const void *> ptrs) {
    if (ldv % Vec<T>::N != 0) return false;
    for (const void *p : ptrs)
        if (p && !aligned16(p)) return false;
    return true;
}

}  // namespace

template <typename T>
cudaError_t launch_mdot(cudaStream_t st, int64_t n, const T *w, const T *V, int64_t ldv, int k, double *partial,
                        double *out, unsigned *counter, const int *done, double *self_nrm, const int *skip) {
    rsv::count_launches(1);
    if (vec_ok<T>(ldv, {w, V}))
        mdot_kernel<T, true><<<kRedBlocks, kRedThreads, 0, st>>>(n, w, V, ldv, k, partial, out, self_nrm, counter,
                                                                 done, skip);
    else
        mdot_kernel<T, false><<<kRedBlocks, kRedThreads, 0, st>>>(n, w, V, ldv, k, partial, out, self_nrm, counter,
                                                                  done, skip);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mdot2(cudaStream_t st, int64_t n, const T *w, const T *u, const T *V, int64_t ldv, int k,
                         double *partial, double *ow, double *ou, unsigned *counter, const int *done) {
    if (k < 1 || k > kMaxRestart + 1) return cudaErrorInvalidValue;
    rsv::count_launches(1);
    if (vec_ok<T>(ldv, {w, u, V}))
        return launch_pdl(mdot2_kernel<T, true>, dim3(kRedBlocks), dim3(kRedThreads), 0, st, n, w, u, V, ldv, k,
                          partial, ow, ou, counter, done);
    return launch_pdl(mdot2_kernel<T, false>, dim3(kRedBlocks), dim3(kRedThreads), 0, st, n, w, u, V, ldv, k, partial,
                      ow, ou, counter, done);
}

template <typename T>
cudaError_t launch_maxpy(cudaStream_t st, int64_t n, const T *base, const T *V, int64_t ldv, int k, const double *c,
                         double sgn, T *out, double *partial, double *nrm, unsigned *counter, const int *done,
                         const int *skip) {
    rsv::count_launches(1);
    if (vec_ok<T>(ldv, {base, V, out}))
        maxpy_kernel<T, true><<<kRedBlocks, kRedThreads, 0, st>>>(n, base, V, ldv, k, c, sgn, out, partial, nrm,
                                                                  counter, done, skip);
    else
        maxpy_kernel<T, false><<<kRedBlocks, kRedThreads, 0, st>>>(n, base, V, ldv, k, c, sgn, out, partial, nrm,
                                                                   counter, done, skip);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_maxpy_mdot(cudaStream_t st, int64_t n, T *w, const T *V, int64_t ldv, int k, const double *c,
                              double *partial, double *proj, double *nrm, unsigned *counter, const int *done) {
    if (k < 1 || k > kFuseMax<T>) return cudaErrorInvalidValue;
    rsv::count_launches(1);
    constexpr int grid = kRedBlocks / 2;  // one CTA per SM: the basis values of a row block live in registers
    if (vec_ok<T>(ldv, {w, V}))
        maxpy_mdot_kernel<T, true><<<grid, kRedThreads, 0, st>>>(n, w, V, ldv, k, c, partial, proj, nrm, counter,
                                                                 done);
    else
        maxpy_mdot_kernel<T, false><<<grid, kRedThreads, 0, st>>>(n, w, V, ldv, k, c, partial, proj, nrm, counter,
                                                                  done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dcgs2_update(cudaStream_t st, int64_t n, T *u, T *w, const T *V, int64_t ldv, int k,
                                const double *cA, const double *cB, const double *cS, const int *done) {
    if (k < 0 || k > kMaxRestart) return cudaErrorInvalidValue;
    rsv::count_launches(1);
    if (vec_ok<T>(ldv, {u, w, V}))
        return launch_pdl(dcgs2_update_kernel<T, true>, dim3(kRedBlocks), dim3(kRedThreads), 0, st, n, u, w, V, ldv,
                          k, cA, cB, cS, done);
    return launch_pdl(dcgs2_update_kernel<T, false>, dim3(kRedBlocks), dim3(kRedThreads), 0, st, n, u, w, V, ldv, k,
                      cA, cB, cS, done);
}

template <typename T>
cudaError_t launch_dot(cudaStream_t st, int64_t n, const T *x, const T *y, double *partial, double *out,
                       unsigned *counter, int sqrt_out, const int *done) {
    rsv::count_launches(1);
    if (vec_ok<T>(Vec<T>::N, {x, y}))
        dot_kernel<T, true><<<kRedBlocks, kRedThreads, 0, st>>>(n, x, y, partial, out, counter, sqrt_out, done);
    else
        dot_kernel<T, false><<<kRedBlocks, kRedThreads, 0, st>>>(n, x, y, partial, out, counter, sqrt_out, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpby(cudaStream_t st, int64_t n, T a, const T *x, T b, const T *y, T *z) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    axpby_kernel<T><<<elementwise_grid(n), 256, 0, st>>>(n, a, x, b, y, z);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_inv(cudaStream_t st, int64_t n, T *x, const double *s, const int *done) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    if (vec_ok<T>(0, {x}))
        scale_inv_kernel<T, true><<<elementwise_grid(n / Vec<T>::N + 1), 256, 0, st>>>(n, x, s, done);
    else
        scale_inv_kernel<T, false><<<elementwise_grid(n), 256, 0, st>>>(n, x, s, done);
    return cudaGetLastError();
}

cudaError_t launch_to_f32_scaled(cudaStream_t st, int64_t n, const double *x, const double *s, float *xf) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    to_f32_scaled<<<elementwise_grid(n), 256, 0, st>>>(n, x, s, xf);
    return cudaGetLastError();
}

cudaError_t launch_add_f32_scaled(cudaStream_t st, int64_t n, const float *df, const double *s, double *x) {
    if (n == 0) return cudaSuccess;
    rsv::count_launches(1);
    add_f32_scaled<<<elementwise_grid(n), 256, 0, st>>>(n, df, s, x);
    return cudaGetLastError();
}

#define RSV_BLAS_INST(T)                                                                                            \
    template cudaError_t launch_mdot<T>(cudaStream_t, int64_t, const T *, const T *, int64_t, int, double *,       \
                                        double *, unsigned *, const int *, double *, const int *);                 \
    template cudaError_t launch_mdot2<T>(cudaStream_t, int64_t, const T *, const T *, const T *, int64_t, int,      \
                                         double *, double *, double *, unsigned *, const int *);                   \
    template cudaError_t launch_maxpy<T>(cudaStream_t, int64_t, const T *, const T *, int64_t, int, const double *, \
                                         double, T *, double *, double *, unsigned *, const int *, const int *);    \
    template cudaError_t launch_maxpy_mdot<T>(cudaStream_t, int64_t, T *, const T *, int64_t, int, const double *,  \
                                              double *, double *, double *, unsigned *, const int *);              \
    template cudaError_t launch_dcgs2_update<T>(cudaStream_t, int64_t, T *, T *, const T *, int64_t, int,           \
                                                const double *, const double *, const double *, const int *);      \
    template cudaError_t launch_dot<T>(cudaStream_t, int64_t, const T *, const T *, double *, double *, unsigned *, \
                                       int, const int *);                                                           \
    template cudaError_t launch_axpby<T>(cudaStream_t, int64_t, T, const T *, T, const T *, T *);                  \
    template cudaError_t launch_scale_inv<T>(cudaStream_t, int64_t, T *, const double *, const int *);
RSV_BLAS_INST(double)
RSV_BLAS_INST(float)

}  // namespace rsv
