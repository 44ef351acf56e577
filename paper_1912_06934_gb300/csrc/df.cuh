// Double-float arithmetic shared by the Krylov kernels of the mixed form.
#pragma once
#include "common.cuh"

// ---- double-float Krylov vectors (mixed form) ----------------------------------------
//
// A Krylov vector v is stored as two FP32 planes, v = hi + lo with |lo| <= ulp(hi)/2
// (about 48 significant bits). Products are formed exactly as p + e
// (e = fma(a, b, -p)) and summed with error-free additions (Knuth TwoSum), so
// dot products and updates run on the FP32 pipe with close-to-FP64 accuracy;
// only O(1) FP64 operations per element remain.

namespace msrsb {

struct DF {
    float hi, lo;
};

// Double-float arithmetic (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2): a value
// is hi + lo with |lo| <= ulp(hi)/2. The _rn intrinsics keep the compiler
// from contracting the error-free transformations into FMAs.
__device__ __forceinline__ DF df_from(double x) {
    float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return DF{s, __fadd_rn(b, -__fadd_rn(s, -a))};
}
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    return DF{s, __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF t = two_sum(a.hi, b.hi);
    return quick_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return quick_two_sum(p, e);
}
// s += a * b in double-float, renormalised after every step so that the low
// word stays within half an ulp of the high word (an unnormalised low word
// collects every rounding error and limits long sums to ~1e-13); the lo*lo
// term is below the format's precision
__device__ __forceinline__ void df_fma_acc(DF &s, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float e = fmaf(ah, bh, -p);
    const DF t = two_sum(s.hi, p);
    s = two_sum(t.hi, __fadd_rn(s.lo, __fadd_rn(t.lo, fmaf(ah, bl, fmaf(al, bh, e)))));
}
__device__ __forceinline__ DF df_shfl_down(DF v, int o) {
    return DF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

}  // namespace msrsb
