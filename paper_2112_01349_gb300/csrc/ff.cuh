// ff.cuh -- float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations: the sum of two floats as a rounded sum plus its exact error
// (Knuth, TAOCP vol. 2, Sec. 4.2.2, after Moller 1965), the same for
// |a| >= |b| in three operations (Dekker 1971), and the product's exact error
// by one fused multiply-add.  Addition and multiplication below follow
// Dekker's double-length procedures (the "sloppy" addition: its error is
// bounded relative to |x| + |y|), and the reciprocal refines the float
// reciprocal by one Newton step, x' = x + x (1 - a x), which doubles its
// correct bits.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so evaluating the cost in
// float-float is several times faster than in FP64 while its error (about
// 1e-13 relative per residual) stays far below the cost changes the LM
// accept test has to resolve.  None of this is used where the library states
// an FP64 result (FP64 problems, mba_evaluate).
#pragma once

#include <cuda_runtime.h>

namespace mba {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_from(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ ff ff_from(float f) { return {f, 0.f}; }
__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = ff_two_sum(x.hi, y.hi);
    return ff_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.hi, -p);  // exact error of the product
    return ff_fast_two_sum(p, e + fmaf(x.hi, y.lo, x.lo * y.hi));
}
__device__ __forceinline__ ff ff_rcp(ff a) {
    const ff x = ff_from(1.f / a.hi);
    const ff r = ff_sub(ff_from(1.f), ff_mul(a, x));  // 1 - a x, small
    return ff_add(x, ff_mul(x, r));
}

}  // namespace mba
