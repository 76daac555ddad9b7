// Double-FP32 ("double-float") arithmetic: a value is hi + lo with two floats,
// |lo| <= ulp(hi)/2, about 48 significant bits. Used for the ray state of the
// bounce kernel (origin, direction, unfolded length) and the reception test,
// where FP32 is too coarse and FP64 is scarce on this GPU. Built from the
// error-free transformations: Knuth's two-sum, Dekker's fast two-sum and the
// FMA-based two-product; division takes two correction steps of the quotient,
// the dot product gathers every lower-order term in one float (the compensated
// dot product of Ogita, Rump and Oishi, 2005).
#pragma once
#include <cuda_runtime.h>

namespace sbr {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// exact split of a double into hi + lo floats
__host__ __device__ __forceinline__ df df_from_double(double x) {
    float h = (float)x;
    return df{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return df{p, __fmaf_rn(a, b, -p)};
}

// a + b with one two-sum on the high words and the low words added in FP32:
// the error is a few units of 2^-48 of the operands' magnitude (not of the
// result's, under cancellation), the absolute accuracy the ray state, the face
// planes and the receiver positions carry in any case
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
// a / b: quotient terms from one reciprocal of b.hi, each correcting the
// residual the previous ones left (computed in double-float); a term only
// needs to be close to the residual's quotient, so the reciprocal's rounding
// does not limit the result
__device__ __forceinline__ df df_div(df a, df b) {
    const float ib = __frcp_rn(b.hi);
    float q1 = a.hi * ib;
    df r = df_sub(a, df_mul_f(b, q1));
    float q2 = r.hi * ib;
    r = df_sub(r, df_mul_f(b, q2));
    float q3 = r.hi * ib;
    df q = fast_two_sum(q1, q2);
    return df_add(q, df{q3, 0.f});
}
// a < b, a <= b on the represented values
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_le(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

struct df3 {
    df x, y, z;
};
__device__ __forceinline__ df3 df3_add(df3 a, df3 b) { return df3{df_add(a.x, b.x), df_add(a.y, b.y), df_add(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_sub(df3 a, df3 b) { return df3{df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_scale(df3 a, df s) { return df3{df_mul(a.x, s), df_mul(a.y, s), df_mul(a.z, s)}; }
// a.b: the three hi*hi products and their two partial sums by error-free
// transformations; their errors, the cross terms hi*lo and lo*hi are summed in
// one float and added once (not symmetric in a, b to the last bit: callers
// keep one argument order per quantity)
__device__ __forceinline__ df df3_dot(df3 a, df3 b) {
    const df px = two_prod(a.x.hi, b.x.hi), py = two_prod(a.y.hi, b.y.hi), pz = two_prod(a.z.hi, b.z.hi);
    const df s1 = two_sum(px.hi, py.hi);
    const df s2 = two_sum(s1.hi, pz.hi);
    float e = __fadd_rn(__fadd_rn(px.lo, py.lo), __fadd_rn(pz.lo, __fadd_rn(s1.lo, s2.lo)));
    e = __fmaf_rn(a.x.hi, b.x.lo, e);
    e = __fmaf_rn(a.x.lo, b.x.hi, e);
    e = __fmaf_rn(a.y.hi, b.y.lo, e);
    e = __fmaf_rn(a.y.lo, b.y.hi, e);
    e = __fmaf_rn(a.z.hi, b.z.lo, e);
    e = __fmaf_rn(a.z.lo, b.z.hi, e);
    return two_sum(s2.hi, e);   // not fast_two_sum: under cancellation |e| may exceed |s2.hi|
}
// a + b c in one pass: the product's high word error-free, its low terms and
// a.lo gathered in FP32 (the accuracy of df_mul followed by df_add)
__device__ __forceinline__ df df_fma(df a, df b, df c) {
    df p = two_prod(b.hi, c.hi);
    p.lo = __fmaf_rn(b.hi, c.lo, p.lo);
    p.lo = __fmaf_rn(b.lo, c.hi, p.lo);
    df s = two_sum(a.hi, p.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, p.lo));
    return fast_two_sum(s.hi, s.lo);
}
// a + b s for vectors a, b and a scalar s
__device__ __forceinline__ df3 df3_fma(df3 a, df3 b, df s) {
    return df3{df_fma(a.x, b.x, s), df_fma(a.y, b.y, s), df_fma(a.z, b.z, s)};
}
__device__ __forceinline__ float3 df3_hi(df3 a) { return make_float3(a.x.hi, a.y.hi, a.z.hi); }

}  // namespace sbr
