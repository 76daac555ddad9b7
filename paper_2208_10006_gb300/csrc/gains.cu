// Complex path gain g_n(f) (Eq. 1, 3, 6-10), one thread per (path, frequency).
//
// Per reflection k (FP32 complex, geometry from the FP64 refinement):
//   eta = eps_r - j sigma / (2 pi f eps0)                         (lossy dielectric)
//   G_TE = (cos - sqrt(eta - sin^2)) / (cos + sqrt(eta - sin^2))
//   G_TM = (eta cos - sqrt(eta - sin^2)) / (eta cos + sqrt(eta - sin^2))
//   rho  = exp(-g/2), g = (4 pi sigma_h cos f / c)^2                (Eq. 6-8)
// applied to the field in the (s, p) basis of that reflection, followed by the
// real 2x2 change to the next reflection's basis; then the Rx projection, the
// Friis amplitude c / (4 pi f L) (Eq. 3), absorption 10^(-gamma L / 20000)
// (Eq. 9) and the dispersion phase -phi (pi/180) L / 1000 (Eq. 10).
#include <algorithm>

#include "sbr_internal.cuh"

namespace sbr {
namespace {

struct cf {
    float re, im;
};
__device__ __forceinline__ cf cmul(cf a, cf b) { return cf{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf cadd(cf a, cf b) { return cf{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf csub(cf a, cf b) { return cf{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cf cdiv(cf a, cf b) {
    float s = fabsf(b.re) + fabsf(b.im);
    float br = b.re / s, bi = b.im / s;
    float d = br * br + bi * bi;
    cf a2{a.re / s, a.im / s};
    return cf{(a2.re * br + a2.im * bi) / d, (a2.im * br - a2.re * bi) / d};
}
// principal square root
__device__ __forceinline__ cf csqrt_(cf z) {
    float r = hypotf(z.re, z.im);
    float x = sqrtf(0.5f * (r + z.re));
    float y = sqrtf(fmaxf(0.5f * (r - z.re), 0.f));
    return cf{x, z.im < 0.f ? -y : y};
}
__device__ __forceinline__ cf cscale(cf a, float s) { return cf{a.re * s, a.im * s}; }

__global__ void k_gains(int64_t P, int32_t F, const int32_t* __restrict__ nb,
                        const int32_t* __restrict__ surf, const double* __restrict__ L,
                        const float* __restrict__ jones, const sbr_material* __restrict__ mats,
                        int32_t S, const double* __restrict__ freqs, const float* __restrict__ gamma,
                        const float* __restrict__ disp, int pol, float2* __restrict__ g,
                        unsigned int* __restrict__ status) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * F) return;
    int64_t p = t / F;
    int32_t fi = (int32_t)(t - p * F);
    const double f = freqs[fi];
    const float* J = jones + p * kJones;
    const int m = nb[p];
    const int pb = pol == SBR_POL_V ? 0 : 2;
    cf b0{__ldg(J + pb), 0.f}, b1{__ldg(J + pb + 1), 0.f};
    const float eps2_scale = (float)(1.0 / (2.0 * kPi * f * kEps0));
    const float kr = (float)(4.0 * kPi * f / kC0);
    for (int k = 0; k < m; ++k) {
        int s = surf[p * kKmax + k];
        if (s < 0 || s >= S) { atomicOr(status, (unsigned)ST_NUMERIC); return; }
        const sbr_material mt = mats[s];
        float c = __ldg(J + 36 + k);
        float s2 = 1.f - c * c;
        cf eta{(float)mt.eps_r, -(float)mt.sigma_s_per_m * eps2_scale};
        cf root = csqrt_(cf{eta.re - s2, eta.im});
        cf cc{c, 0.f};
        cf te = cdiv(csub(cc, root), cadd(cc, root));
        cf ec = cscale(eta, c);
        cf tm = cdiv(csub(ec, root), cadd(ec, root));
        float gk = kr * (float)mt.rough_m * c;
        float rho = expf(-0.5f * gk * gk);
        b0 = cscale(cmul(te, b0), rho);
        b1 = cscale(cmul(tm, b1), rho);
        if (k + 1 < m) {
            const float* M = J + 4 + 4 * k;
            cf n0 = cadd(cscale(b0, M[0]), cscale(b1, M[1]));
            cf n1 = cadd(cscale(b0, M[2]), cscale(b1, M[3]));
            b0 = n0;
            b1 = n1;
        }
    }
    const float* cv = J + 32 + pb;
    cf proj = cadd(cscale(b0, cv[0]), cscale(b1, cv[1]));
    const double Lp = L[p];
    float amp = (float)(kC0 / (4.0 * kPi * f * Lp));
    float att = gamma ? exp10f(-gamma[fi] * (float)Lp * (1.0f / 20000.0f)) : 1.f;
    float ph = disp ? -disp[fi] * (float)(kPi / 180.0 * Lp / 1000.0) : 0.f;
    float sn, cs;
    sincosf(ph, &sn, &cs);
    cf v = cmul(cscale(cf{cs, sn}, amp * att), proj);
    g[t] = make_float2(v.re, v.im);
}

}  // namespace

sbr_status gains_run(const sbr_path_list* pl, const sbr_material* mats, int32_t S,
                     const double* freqs, int32_t F, const float* gamma, const float* disp,
                     int32_t pol, float2* g, cudaStream_t s) {
    int64_t n = pl->P * (int64_t)F;
    if (n == 0) return SBR_OK;
    unsigned int* status;
    SBR_TRY(dalloc_n(&status, 1, s));
    SBR_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
    k_gains<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pl->P, F, pl->nb, pl->surf, pl->L, pl->jones,
                                                          mats, S, freqs, gamma, disp, pol, g, status);
    SBR_TRY_CUDA(cudaGetLastError());
    dfree(status, s);
    return SBR_OK;
}

}  // namespace sbr
