// Double-float arithmetic for the mixed-precision Krylov matvec.
//
// A value is hi + lo, two FP32 numbers with |lo| <= ulp(hi) / 2 (about 48
// significand bits).  Products use the FMA form of the exact product
// (p = a b, e = fma(a, b, -p) is exact), sums Knuth's TwoSum (Dekker 1971,
// Knuth TAOCP vol. 2, 4.2.2); the result is renormalised after every
// operation.  Every operation goes through the _rn intrinsics, which the
// compiler never contracts into FMAs, so the error-free steps stay exact.
// On this part FP32 issues 64 times faster than FP64, which makes a handful of
// FP32 operations per double-float operation the cheaper way to carry ~1e-14
// relative accuracy.
#pragma once
#include <cuda_runtime.h>

struct df64 {
    float hi, lo;
};

__device__ __forceinline__ df64 df_make(float hi, float lo) {
    df64 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// nearest double-float to x (FP64 operations: for set-up, not inner loops)
__device__ __forceinline__ df64 df_from_double(double x) {
    const float h = __double2float_rn(x);
    return df_make(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df64 df_from_float2(float2 v) { return df_make(v.x, v.y); }
__device__ __forceinline__ float2 df_to_float2(df64 a) { return make_float2(a.hi, a.lo); }

__device__ __forceinline__ df64 df_neg(df64 a) { return df_make(-a.hi, -a.lo); }

// a + b: TwoSum of the high parts, the low parts added to its error, renormalised
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, t);
    return df_make(h, __fsub_rn(t, __fsub_rn(h, s)));
}

// a b: exact product of the high parts plus the cross terms, renormalised
__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    const float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    const float h = __fadd_rn(p, t);
    return df_make(h, __fsub_rn(t, __fsub_rn(h, p)));
}

__device__ __forceinline__ df64 df_shfl_xor(df64 a, int o) {
    return df_make(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
}
