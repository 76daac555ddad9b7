// Operands of the tensor-core H(f) synthesis (Eq. 13-14), shared by the
// single-receiver and the batched forms so that both compute them with the
// same arithmetic (and therefore give bit-identical H for the same paths).
//
// Layout, for the Pr reflected paths of one receiver padded to Pp (a multiple
// of 8; padded entries are zero):
//   w   [F][Pp]  float2  g_n(f) exp(-j 2 pi f L_n / c), reflected paths only
//   wl  [F]      float2  the same for the LoS path (zero when there is none)
//   sc  [F]      float   FP16 form: the power of two that brings
//                        max_n max(|Re w|, |Im w|) into [1/2, 1) (1 if all zero)
//   dtT [Pp/4][Nt][4] float   |T_p - P1| - |T_0 - P1|   (P1 first interaction point)
//   drT [Pp/4][Nr][4] float   |R_q - Pm| - |R_0 - Pm|   (Pm last interaction point)
//   dl  [Nr][Nt] float   |T_p - R_q| - |T_0 - R_0|
// (the delay tables in groups of 4 paths, element-major within a group, so
// that consecutive threads, on consecutive elements, read consecutive 16-byte
// groups)
#pragma once
#include "sbr_internal.cuh"

namespace sbr {

constexpr double kInvC0 = 1.0 / kC0;

// g exp(-j 2 pi f L / c). The phase f L / c (up to ~1e6 cycles at THz) is
// reduced exactly in FP64 to its fraction r in [0, 1); r = hi + lo with hi the
// FP32 rounding of r and |lo| <= 2^-25; exp(-j 2 pi r) = exp(-j 2 pi hi)
// (1 - j 2 pi lo) to second order in lo (< 1e-13), with the FP32 sine and
// cosine of pi x (sincospif) for the hi part. FP64 is used for 7 operations
// only: this GPU's FP64 rate is a small fraction of its FP32 rate.
//
// Every operation is written with an explicit rounding intrinsic, so that the
// compiler cannot contract a multiply and an add differently in the kernels
// that share these functions (their results must agree bit for bit).
__device__ __forceinline__ float2 synth_weight(float2 g, double f, double L) {
    const double cyc = __dmul_rn(__dmul_rn(f, L), kInvC0);
    const double r = __dsub_rn(cyc, floor(cyc));
    const float hi = __double2float_rn(r);
    const float lo = __double2float_rn(__dsub_rn(r, (double)hi));
    float s, c;
    sincospif(__fmul_rn(-2.0f, hi), &s, &c);
    const float d = __fmul_rn(-6.283185307179586f, lo);   // exp(j d) ~ 1 + j d
    const float cr = __fmaf_rn(-s, d, c), ci = __fmaf_rn(c, d, s);
    return make_float2(__fmaf_rn(g.x, cr, __fmul_rn(-g.y, ci)), __fmaf_rn(g.x, ci, __fmul_rn(g.y, cr)));
}

// the FP16 form's per-frequency scale from the largest weight component
__device__ __forceinline__ float synth_scale(float m) {
    if (!(m > 0.f)) return 1.f;
    int e;
    frexpf(m, &e);
    return ldexpf(1.f, -e);
}

// |a - b| in FP64 with a fixed operation sequence
__device__ __forceinline__ double dist_rn(d3 a, d3 b) {
    const double x = __dsub_rn(a.x, b.x), y = __dsub_rn(a.y, b.y), z = __dsub_rn(a.z, b.z);
    return __dsqrt_rn(__fma_rn(z, z, __fma_rn(y, y, __dmul_rn(x, x))));
}

// element delay |E - P| - ref, ref = |E0 - P| = dist_rn(E0, P) computed once
// per path (FP64, then rounded to FP32)
__device__ __forceinline__ float el_delay(const double* elem, d3 P, double ref) {
    return __double2float_rn(__dsub_rn(dist_rn(ld3(elem), P), ref));
}

}  // namespace sbr
