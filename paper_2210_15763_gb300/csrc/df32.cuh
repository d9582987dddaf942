// Float-float ("double-FP32") numbers for the polish stage of the
// mixed-precision solver: a value is the unevaluated sum hi + lo of two FP32
// numbers, about 48 significant bits.  GB300 runs FP32 arithmetic at many
// times its FP64 rate, so the polish's SpMM and Gram-Schmidt products run on
// the FP32 pipes.
//
// The error-free transformations are the classical ones: Knuth's TwoSum
// (s + e = a + b exactly, six operations) and the FMA form of Dekker's
// TwoProduct (p + e = a * b exactly).  Sums of many products are kept
// unnormalised (the low parts are summed in FP32 and the pair is normalised
// only when stored), which keeps the error near 2^-48 of the sum of the
// absolute products.
#pragma once

#include <cuda_runtime.h>

namespace bbl {
namespace dfm {

struct __align__(8) df32 {
    float hi, lo;
    df32() = default;
    __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df32(float h) : hi(h), lo(0.0f) {}
    __host__ __device__ constexpr df32(int h) : hi((float)h), lo(0.0f) {}
    // nearest pair to an FP64 value: hi = fl32(x), lo = fl32(x - hi)
    __host__ __device__ explicit df32(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// normalised pair from an unnormalised one
__device__ __forceinline__ df32 renorm(float h, float l) {
    float s, e;
    two_sum(h, l, s, e);
    return df32(s, e);
}

// c + a * b, result unnormalised (accumulator form)
__device__ __forceinline__ df32 fma(df32 a, df32 b, df32 c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    return df32(s, __fadd_rn(c.lo, __fadd_rn(e, t)));
}

// c + h * v with an FP32 factor h (an SpMM's matrix value)
__device__ __forceinline__ df32 fma(float h, df32 v, df32 c) {
    const float p = __fmul_rn(h, v.hi);
    float e = __fmaf_rn(h, v.hi, -p);
    e = __fmaf_rn(h, v.lo, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    return df32(s, __fadd_rn(c.lo, __fadd_rn(e, t)));
}

__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
    float s, t;
    two_sum(a.hi, b.hi, s, t);
    return renorm(s, __fadd_rn(t, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + df32(-b.hi, -b.lo); }

__device__ __forceinline__ df32& operator+=(df32& a, df32 b) {
    a = a + b;
    return a;
}

__device__ __forceinline__ df32 shfl_xor(unsigned mask, df32 v, int off) {
    return df32(__shfl_xor_sync(mask, v.hi, off), __shfl_xor_sync(mask, v.lo, off));
}

}  // namespace dfm

using dfm::df32;

template <typename T>
struct is_df32 {
    static constexpr bool value = false;
};
template <>
struct is_df32<df32> {
    static constexpr bool value = true;
};

// xor shuffle for the accumulator types of the kernels
template <typename T>
__device__ __forceinline__ T shfl_xor_any(unsigned mask, T v, int off) {
    if constexpr (is_df32<T>::value) return dfm::shfl_xor(mask, v, off);
    else return __shfl_xor_sync(mask, v, off);
}

}  // namespace bbl

namespace bbl {
namespace dfm {

// normalised float-float operations for the sequential recurrences of the
// Ritz solve (where FP64 would cost one 64-cycle issue slot per instruction)
__device__ __forceinline__ df32 dmul(df32 a, df32 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return renorm(p, e);
}

// c + a * b, normalised
__device__ __forceinline__ df32 dfma(df32 a, df32 b, df32 c) {
    const df32 t = fma(a, b, c);
    return renorm(t.hi, t.lo);
}

__device__ __forceinline__ df32 dneg(df32 a) { return df32(-a.hi, -a.lo); }

// 1 / a: FP32 seed and one Newton step in float-float (about 46 bits)
__device__ __forceinline__ df32 drcp(df32 a) {
    const float r0 = __frcp_rn(a.hi);
    // e = 1 - a * r0 (exact product terms, then the float-float difference)
    const df32 ar = dmul(a, df32(r0));
    const df32 e = df32(1.0f) - ar;
    return dfma(df32(r0), e, df32(r0));
}

}  // namespace dfm
}  // namespace bbl
