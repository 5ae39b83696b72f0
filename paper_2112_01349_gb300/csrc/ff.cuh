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
//
// The header also compiles as plain C++ (host functions only), so that the
// error bounds can be checked on the host against exact rational arithmetic;
// such a build must keep the compiler from contracting a*b + c into an FMA
// (-ffp-contract=off), which would break the error-free transformations.
// On the device every plain product is rounded by __fmul_rn, which the
// compiler never merges into an FMA, and the others are explicit FMAs.
// Host and device builds therefore perform the same IEEE operations.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define MBA_FF __host__ __device__ __forceinline__
#else
#define MBA_FF inline
#endif

namespace mba {

struct ff {
    float hi, lo;
};

MBA_FF float ff_mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

MBA_FF ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
MBA_FF ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
MBA_FF ff ff_from(double d) {
    const float h = static_cast<float>(d);  // round to nearest
    return {h, static_cast<float>(d - (double)h)};
}
MBA_FF ff ff_from(float f) { return {f, 0.f}; }
MBA_FF double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }
MBA_FF ff ff_add(ff x, ff y) {
    const ff s = ff_two_sum(x.hi, y.hi);
    return ff_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
MBA_FF ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
MBA_FF ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
MBA_FF ff ff_mul(ff x, ff y) {
    const float p = ff_mul_rn(x.hi, y.hi);
    const float e = fmaf(x.hi, y.hi, -p);  // exact error of the product
    return ff_fast_two_sum(p, e + fmaf(x.hi, y.lo, ff_mul_rn(x.lo, y.hi)));
}
MBA_FF ff ff_rcp(ff a) {
    const ff x = ff_from(1.f / a.hi);
    const ff r = ff_sub(ff_from(1.f), ff_mul(a, x));  // 1 - a x, small
    return ff_add(x, ff_mul(x, r));
}

}  // namespace mba
