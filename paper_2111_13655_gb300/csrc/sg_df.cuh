// Double-float ("double-word") numbers for the FP64-class contraction type:
// a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits, computed on the FP32 pipes
// (which GB300 runs at 73 times its FP64 rate).  Host and device code: the
// host builds the tables in this form, and the CPU tests check the error
// bounds of these exact functions.
//
// Building blocks (error-free transformations, with u = 2^-24):
//   two_sum(a, b)       s + e = a + b exactly, s = fl(a + b)        (Knuth)
//   fast_two_sum(a, b)  the same for |a| >= |b|, three operations   (Dekker)
//   two_prod(a, b)      p + e = a * b exactly with one FMA
// Operations on double-floats:
//   df_mul(x, y)        product: the exact product of the high parts, the
//                       two cross terms added by FMA, renormalised (the lo*lo
//                       term, below u^2 of the result, is dropped); relative
//                       error below 4u^2.
//   df_fma(x, y, c)     c + x * y as one step of a compensated dot product:
//                       the product as in df_mul, its high part added to c's
//                       high part by two_sum, the two low parts and the
//                       rounding error summed in FP32 (12 FP32 instructions;
//                       not renormalised unless SG_DF_RENORM).  The error is
//                       within a few u^2 (|x y| + |c|): the sum is as
//                       accurate as if computed with 2^-48 and rounded.
// From double: hi = fl32(d), lo = fl32(d - hi); hi + lo equals d to 2^-48
// relative (d - hi is exact in FP64).
#pragma once

#include <cmath>

#if !defined(__CUDACC__) && defined(__has_include)
#if __has_include(<cuda_runtime.h>)
#include <cuda_runtime.h>
#endif
#endif
// plain C++ (the CPU tests of these functions): the CUDA qualifiers vanish
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#ifndef __align__
#define __align__(n) alignas(n)
#endif

// 1: renormalise after every multiply-add (three more FP32 instructions)
#ifndef SG_DF_RENORM
#define SG_DF_RENORM 0
#endif

namespace sg {

struct __align__(8) df2 {
    float hi, lo;
    df2() = default;
    __host__ __device__ constexpr df2(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df2(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ df2(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

namespace dfops {

// Single-rounding FP32 operations that the compiler may not fuse or reorder
// (a product contracted into a later addition would break the exact
// transformations below).
__host__ __device__ inline float add(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ inline float sub(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ inline float mul(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ inline float fma32(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}

// s + e = a + b exactly
__host__ __device__ inline void two_sum(float a, float b, float &s, float &e)
{
    s = add(a, b);
    const float ap = sub(s, b);
    const float bp = sub(s, ap);
    e = add(sub(a, ap), sub(b, bp));
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__host__ __device__ inline void fast_two_sum(float a, float b, float &s, float &e)
{
    s = add(a, b);
    e = sub(b, sub(s, a));
}

}  // namespace dfops

__host__ __device__ inline df2 df_mul(df2 x, df2 y)
{
    const float p = dfops::mul(x.hi, y.hi);
    float e = dfops::fma32(x.hi, y.hi, -p);  // p + e = x.hi * y.hi exactly
    e = dfops::fma32(x.hi, y.lo, e);
    e = dfops::fma32(x.lo, y.hi, e);
    df2 r;
    dfops::fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

__host__ __device__ inline df2 df_fma(df2 x, df2 y, df2 c)
{
    const float p = dfops::mul(x.hi, y.hi);
    float e = dfops::fma32(x.hi, y.hi, -p);
    e = dfops::fma32(x.hi, y.lo, e);
    e = dfops::fma32(x.lo, y.hi, e);
    float s, t;
    dfops::two_sum(c.hi, p, s, t);  // s + t = c.hi + p exactly
    t = dfops::add(t, dfops::add(e, c.lo));
#if SG_DF_RENORM
    df2 r;
    dfops::fast_two_sum(s, t, r.hi, r.lo);
    return r;
#else
    // not renormalised: (s, t) holds the same value, t possibly above
    // ulp(s) / 2; every consumer takes it as the sum hi + lo (the next
    // multiply-add exactly so, the exact fixed-point conversion of hi and lo
    // too, and a product with an extra error of u |x| |t|: a few u^2 |x s|
    // unless s came from a cancellation, where it is u^2 of the cancelled
    // terms as in a compensated dot product)
    return df2(s, t);
#endif
}

__host__ __device__ inline df2 operator*(df2 x, df2 y) { return df_mul(x, y); }
__host__ __device__ inline df2 &operator*=(df2 &x, df2 y) { return x = df_mul(x, y); }

}  // namespace sg
