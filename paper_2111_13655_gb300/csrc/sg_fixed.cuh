// Exact fixed-point accumulation of the compact result (device code shared by
// the kernels).  A value r is added as an integer multiple of 2^E, held in
// kAccDigits signed 32-bit digits stored in int64 words: integer additions are
// exact and associative, so the sum does not depend on the order of additions.
#pragma once

#include "sg_df.cuh"
#include "sg_internal.h"

namespace sg {
namespace fx {

// Adds coef * r (r = +-mant * 2^e2) to the fixed-point accumulator acc[0..3]
// in units of 2^E.  Integer arithmetic only: the result is exact up to the
// rounding of values below 2^E, and independent of the order of additions.
static __device__ __forceinline__ void fx_add(unsigned long long *acc, unsigned long long mant, int e2, bool neg,
                                       int coef, int E, int *err)
{
    if (mant == 0 || coef == 0) return;
    if (coef < 0) { neg = !neg; coef = -coef; }
    const int sh = e2 - E;
    if (mant < (1ull << 24) && sh >= 0 && sh <= 30) {
        // FP32 values: the exact product fits 56 bits and, shifted, 86 bits: two
        // 64-bit halves, digits taken from them directly
        const unsigned long long pm = mant * (unsigned)coef;       // < 2^56
        const unsigned long long lo = pm << sh;                    // bits 0..63
        const unsigned long long hi = sh ? pm >> (64 - sh) : 0ull; // bits 64..127
        const unsigned long long d[4] = {lo & 0xFFFFFFFFull, lo >> 32, hi & 0xFFFFFFFFull, hi >> 32};
#pragma unroll
        for (int i = 0; i < kAccDigits; i++)
            if (d[i]) atomicAdd(acc + i, neg ? (unsigned long long)(-(long long)d[i]) : d[i]);
        return;
    }
    const unsigned __int128 Pm = (unsigned __int128)mant * (unsigned)coef;  // < 2^85, exact
    unsigned __int128 F;
    if (sh >= 0) {
        if (sh > 126 || (Pm >> (126 - sh)) != 0) {  // would leave the 127-bit range
            if (err) atomicCAS(err, 0, 200);
            return;
        }
        F = Pm << sh;
    } else {
        const int rs = -sh;
        if (rs >= 127) return;                        // below 2^E: rounds to zero
        F = (Pm + ((unsigned __int128)1 << (rs - 1))) >> rs;
    }
#pragma unroll
    for (int i = 0; i < kAccDigits; i++) {
        const unsigned long long d = (unsigned long long)(F >> (32 * i)) & 0xFFFFFFFFull;
        if (d) atomicAdd(acc + i, neg ? (unsigned long long)(-(long long)d) : d);
    }
}

static __device__ __forceinline__ void fx_add_real(unsigned long long *acc, double r, int coef, int E, int *err)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(r);
    int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
    if (ex == 0x7FF) { if (err) atomicCAS(err, 0, 201); return; }
    if (ex == 0) ex = 1; else mant |= 1ull << 52;
    fx_add(acc, mant, ex - 1075, (bits >> 63) != 0, coef, E, err);
}

static __device__ __forceinline__ void fx_add_real(unsigned long long *acc, float r, int coef, int E, int *err)
{
    const unsigned bits = (unsigned)__float_as_uint(r);
    int ex = (int)((bits >> 23) & 0xFF);
    unsigned long long mant = bits & 0x7FFFFFu;
    if (ex == 0xFF) { if (err) atomicCAS(err, 0, 201); return; }
    if (ex == 0) ex = 1; else mant |= 1ull << 23;
    fx_add(acc, mant, ex - 150, (bits >> 31) != 0, coef, E, err);
}

// E (the exponent of the accumulators' unit) of vector v from max|x_v|
static __device__ __forceinline__ int lsb_exponent(long long maxbits, int below = kAccLsbBelowMax)
{
    const int ex = (int)((maxbits >> 52) & 0x7FF);
    if (maxbits == 0) return -1000;
    return (ex - 1022) - below;  // max|x| < 2^(ex-1022)
}

// FP32 contributions into one signed 64-bit word in units of 2^E: coef * r is
// rounded to the nearest unit (half up) and added with one integer atomic.
// With E = exponent(max|x|) - 40 a single contribution stays below 2^62 units
// (|coef * r| < 2^22 max|x|; larger ones set error 202), the rounding of each
// is at most 2^(E-1), and sums wrap modulo 2^64 harmlessly: the final value
// (|y| far below 2^23 max|x|) is exact up to those roundings, in any order.
static __device__ __forceinline__ void fx_add_w1(unsigned long long *acc, float r, int coef, int E, int *err)
{
    const unsigned bits = (unsigned)__float_as_uint(r);
    int ex = (int)((bits >> 23) & 0xFF);
    unsigned long long mant = bits & 0x7FFFFFu;
    if (ex == 0xFF) { if (err) atomicCAS(err, 0, 201); return; }
    if (ex == 0) ex = 1; else mant |= 1ull << 23;
    if (mant == 0 || coef == 0) return;
    bool neg = (bits >> 31) != 0;
    if (coef < 0) { neg = !neg; coef = -coef; }
    const unsigned long long pm = mant * (unsigned)coef;  // < 2^33, exact
    const int sh = (ex - 150) - E;
    unsigned long long v;
    if (sh >= 0) {
        if (sh > 29) { if (err) atomicCAS(err, 0, 202); return; }
        v = pm << sh;
    } else {
        const int rs = -sh;
        if (rs > 33) return;  // below half a unit: rounds to zero
        v = (pm + (1ull << (rs - 1))) >> rs;
    }
    if (v) atomicAdd(acc, neg ? (unsigned long long)(-(long long)v) : v);
}

// The accumulator format of a contraction type: FP64 four 32-bit digits
// (exact), FP32 one word (above).
template <typename T> struct Acc;
template <> struct Acc<double> {
    static constexpr int words = kAccDigits;
    static __device__ __forceinline__ int unit(long long mb) { return lsb_exponent(mb); }
    static __device__ __forceinline__ void add_unit(unsigned long long *a, double r, int coef, int E, int *err)
    {
        fx_add_real(a, r, coef, E, err);
    }
    static __device__ __forceinline__ void add(unsigned long long *a, double r, int coef, long long mb, int *err)
    {
        add_unit(a, r, coef, unit(mb), err);
    }
};
// Double-float contributions: the FP64 accumulator format; the high and low
// parts are added as two exact contributions (integer arithmetic only).
template <> struct Acc<df2> {
    static constexpr int words = kAccDigits;
    static __device__ __forceinline__ int unit(long long mb) { return lsb_exponent(mb); }
    static __device__ __forceinline__ void add_unit(unsigned long long *a, df2 r, int coef, int E, int *err)
    {
        fx_add_real(a, r.hi, coef, E, err);
        fx_add_real(a, r.lo, coef, E, err);
    }
    static __device__ __forceinline__ void add(unsigned long long *a, df2 r, int coef, long long mb, int *err)
    {
        add_unit(a, r, coef, unit(mb), err);
    }
};
template <> struct Acc<float> {
    static constexpr int words = 1;
    static __device__ __forceinline__ int unit(long long mb) { return lsb_exponent(mb, kAcc32LsbBelowMax); }
    static __device__ __forceinline__ void add_unit(unsigned long long *a, float r, int coef, int E, int *err)
    {
        fx_add_w1(a, r, coef, E, err);
    }
    static __device__ __forceinline__ void add(unsigned long long *a, float r, int coef, long long mb, int *err)
    {
        add_unit(a, r, coef, unit(mb), err);
    }
};


}  // namespace fx
}  // namespace sg
