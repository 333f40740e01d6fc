// Double-float value type for the reaction passes that fix the answer in
// mixed precision (F(U) of the predictor and of the Newton residual).
//
// A value is the unevaluated sum hi + lo of two FP32 numbers, carrying about
// 48 significand bits.  The kernels of the reaction term are templates over
// their element type; with T = dfloat they run the same code in double-float
// arithmetic:
//   a * b  exact product of the high parts (p = a.hi b.hi, e = fma(a.hi,
//          b.hi, -p) is exact) plus the cross terms a.hi b.lo + a.lo b.hi
//          folded into e -- 4 FP32 operations;
//   a + b  Knuth's TwoSum of the high parts (Knuth, TAOCP vol. 2, 4.2.2;
//          Dekker 1971), the low parts added to its rounding error --
//          8 FP32 operations.
// Results are not renormalised inside the loops: the pair stays a correct
// representation of the value (|lo| grows to a few ulps of hi at most
// between renormalisations), and TwoSum is exact whatever the relative size
// of its arguments, so skipping the 3-operation renormalisation only moves
// the last bits.  Conversions to double sum the pair in FP64.  Every step
// goes through the _rn intrinsics, which the compiler never contracts or
// reassociates, so the error-free steps stay exact.
//
// sizeof(dfloat) == sizeof(double): the double-float passes use the FP64
// work buffers and fiber plans unchanged.  On this part FP32 issues ~64x
// faster than FP64, so ~12 FP32 operations per multiply-add are still the
// cheaper way to ~1e-14 relative accuracy.
#pragma once
#include <cuda_runtime.h>

struct __align__(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    // exact for integers of magnitude below 2^24
    __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.0f) {}
    // nearest pair to x: hi = fl32(x), lo = fl32(x - hi)
    __host__ __device__ dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};
static_assert(sizeof(dfloat) == 8, "dfloat has the size of a double");

#ifdef __CUDACC__
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dfloat(p, e);
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return dfloat(s, __fadd_rn(err, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }

// renormalised pair: |lo| <= ulp(hi) / 2
__device__ __forceinline__ dfloat df_norm(dfloat a) {
    const float h = __fadd_rn(a.hi, a.lo);
    return dfloat(h, __fsub_rn(a.lo, __fsub_rn(h, a.hi)));
}

__device__ __forceinline__ double df_value(dfloat a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float df_float(dfloat a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ dfloat df_split(double x) {
    const float h = __double2float_rn(x);
    return dfloat(h, __double2float_rn(x - (double)h));
}

// read through volatile pointers (the element re-read at every use)
template <typename T>
__device__ __forceinline__ T volatile_read(const T* p) {
    return *reinterpret_cast<const volatile T*>(p);
}
template <>
__device__ __forceinline__ dfloat volatile_read<dfloat>(const dfloat* p) {
    const volatile float* f = reinterpret_cast<const volatile float*>(p);
    return dfloat(f[0], f[1]);
}
#endif
