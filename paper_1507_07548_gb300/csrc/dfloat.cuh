// Double-float arithmetic: a value carried as an unevaluated sum h + l of two
// FP32 numbers (about 44 significant bits), built from the error-free
// transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the FMA-based exact
// product.  Used where one FP32 rounding is too coarse: the site pairs at close
// contact, whose r^-12 terms carry the large, strongly cancelling part of the
// molecular virial of a dense polar liquid.
#pragma once
#include <cuda_runtime.h>

namespace dfl {

struct df {
    float h, l;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly (the FMA gives the rounding error of the product)
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df add(df x, df y) {
    df s = two_sum(x.h, y.h);
    s.l = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df neg(df x) { return {-x.h, -x.l}; }

__device__ __forceinline__ df mul(df x, df y) {
    df p = two_prod(x.h, y.h);
    p.l = __fmaf_rn(x.h, y.l, p.l);
    p.l = __fmaf_rn(x.l, y.h, p.l);
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ df mul_f(df x, float f) {
    df p = two_prod(x.h, f);
    p.l = __fmaf_rn(x.l, f, p.l);
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ df sqr(df x) {
    df p = two_prod(x.h, x.h);
    p.l = __fmaf_rn(__fadd_rn(x.h, x.h), x.l, p.l);
    return fast_two_sum(p.h, p.l);
}

// 1 / x: the FP32 reciprocal refined by one Newton step on the exact residual
// 1 - x y (x.h y - 1 is exact through the FMA when y is within an ulp of 1/x.h)
__device__ __forceinline__ df rcp(df x) {
    const float y = __frcp_rn(x.h);
    float r = __fmaf_rn(-x.h, y, 1.0f);
    r = __fmaf_rn(-x.l, y, r);
    return fast_two_sum(y, __fmul_rn(y, r));
}

}  // namespace dfl
