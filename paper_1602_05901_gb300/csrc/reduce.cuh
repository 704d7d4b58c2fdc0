// Internal: FP64-accurate accumulation and 16-byte vector helpers shared by
// the reduction kernels (blas.cu, batch.cu).
#pragma once

#include "common.cuh"

namespace rsv {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of products, FP64-accurate.
template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);         // a*b = p + pe exactly
        const float s = __fadd_rn(hi, p);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));  // hi + p = s + err
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, pe));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// A partial sum in its accumulator's form, for the warp reduction trees: an FP64
// value, or a double-float pair (FP32 hi + lo) whose additions are Knuth
// two-sums on the FP32 pipes.  GB300 runs FP64 arithmetic at a small fraction of
// its FP32 rate, so FP32 vectors' sums stay off the FP64 pipe until one value per
// warp is widened.  A double-float addition keeps about 46 bits of the sum.
template <typename T> struct Part;
template <> struct Part<double> {
    double s;
    __device__ __forceinline__ static Part of(const Acc<double> &a) { return {a.s}; }
    __device__ __forceinline__ static Part zero() { return {0.0}; }
    __device__ __forceinline__ Part xor_shfl(int o) const { return {__shfl_xor_sync(0xffffffffu, s, o)}; }
    __device__ __forceinline__ void add(const Part &b) { s += b.s; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Part<float> {
    float hi, lo;
    __device__ __forceinline__ static Part of(const Acc<float> &a) { return {a.hi, a.lo}; }
    __device__ __forceinline__ static Part zero() { return {0.f, 0.f}; }
    __device__ __forceinline__ Part xor_shfl(int o) const {
        return {__shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o)};
    }
    __device__ __forceinline__ void add(const Part &b) {
        // two-sums of the high and of the low parts, then two renormalisations
        const float s = __fadd_rn(hi, b.hi);
        const float sb = __fsub_rn(s, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, sb)), __fsub_rn(b.hi, sb));
        const float t = __fadd_rn(lo, b.lo);
        const float tb = __fsub_rn(t, lo);
        const float f = __fadd_rn(__fsub_rn(lo, __fsub_rn(t, tb)), __fsub_rn(b.lo, tb));
        e = __fadd_rn(e, t);
        const float h = __fadd_rn(s, e);
        e = __fadd_rn(__fsub_rn(e, __fsub_rn(h, s)), f);
        hi = __fadd_rn(h, e);
        lo = __fsub_rn(e, __fsub_rn(hi, h));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T> struct Vec;
template <> struct Vec<float> {
    using V = float4;
    static constexpr int N = 4;
    __device__ __forceinline__ static float get(const float4 &v, int q) {
        return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
    }
    __device__ __forceinline__ static void set(float4 &v, int q, float x) {
        if (q == 0) v.x = x; else if (q == 1) v.y = x; else if (q == 2) v.z = x; else v.w = x;
    }
};
template <> struct Vec<double> {
    using V = double2;
    static constexpr int N = 2;
    __device__ __forceinline__ static double get(const double2 &v, int q) { return q == 0 ? v.x : v.y; }
    __device__ __forceinline__ static void set(double2 &v, int q, double x) {
        if (q == 0) v.x = x; else v.y = x;
    }
};

}  // namespace rsv
