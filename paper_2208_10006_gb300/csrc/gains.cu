// Complex path gain g_n(f) (Eq. 1, 3, 6-10), one thread per (path, frequency).
//
// Per reflection k (FP64 complex):
//   eta = eps_r - j sigma / (2 pi f eps0)                         (lossy dielectric)
//   G_TE = (cos - sqrt(eta - sin^2)) / (cos + sqrt(eta - sin^2))
//   G_TM = (eta cos - sqrt(eta - sin^2)) / (eta cos + sqrt(eta - sin^2))
//   rho  = exp(-g/2), g = (4 pi sigma_h cos f / c)^2                (Eq. 6-8)
// applied to the field in the (s, p) basis of that reflection, followed by the
// real 2x2 change to the next reflection's basis; then the Rx projection, the
// Friis amplitude c / (4 pi f L) (Eq. 3), absorption 10^(-gamma L / 20000)
// (Eq. 9) and the dispersion phase -phi (pi/180) L / 1000 (Eq. 10).
// FP64 because the co-polar projection of a multi-bounce field can cancel to
// 1e-5 of the field, below which FP32 rounding alone exceeds a 1e-4 relative
// error on the gain; the work is P x F, negligible next to the trace.
#include <algorithm>

#include "sbr_internal.cuh"

namespace sbr {
namespace {

struct cd {
    double re, im;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return cd{a.re * s, a.im * s}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    double s = fabs(b.re) + fabs(b.im);
    double br = b.re / s, bi = b.im / s;
    double d = br * br + bi * bi;
    double ar = a.re / s, ai = a.im / s;
    return cd{(ar * br + ai * bi) / d, (ai * br - ar * bi) / d};
}
// principal square root
__device__ __forceinline__ cd csqrt_(cd z) {
    double r = hypot(z.re, z.im);
    double x = sqrt(0.5 * (r + z.re));
    double y = sqrt(fmax(0.5 * (r - z.re), 0.0));
    return cd{x, z.im < 0.0 ? -y : y};
}

__global__ void k_gains(int64_t P, int32_t F, const int32_t* __restrict__ nb,
                        const int32_t* __restrict__ surf, const double* __restrict__ L,
                        const double* __restrict__ jones, const sbr_material* __restrict__ mats,
                        int32_t S, const double* __restrict__ freqs, const float* __restrict__ gamma,
                        const float* __restrict__ disp, int pol, float2* __restrict__ g) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * F) return;
    int64_t p = t / F;
    int32_t fi = (int32_t)(t - p * F);
    const double f = freqs[fi];
    const double* J = jones + p * kJones;
    const int m = nb[p];
    const int pb = pol == SBR_POL_V ? 0 : 2;
    cd b0{J[pb], 0.0}, b1{J[pb + 1], 0.0};
    const double eps2_scale = 1.0 / (2.0 * kPi * f * kEps0);
    const double kr = 4.0 * kPi * f / kC0;
    for (int k = 0; k < m; ++k) {
        int s = surf[p * kKmax + k];
        if (s < 0 || s >= S) {  // not reachable: the host checks S covers every surface id
            g[t] = make_float2(NAN, NAN);
            return;
        }
        const sbr_material mt = mats[s];
        double c = J[36 + k];
        double s2 = 1.0 - c * c;
        cd eta{mt.eps_r, -mt.sigma_s_per_m * eps2_scale};
        cd root = csqrt_(cd{eta.re - s2, eta.im});
        cd cc{c, 0.0};
        cd te = cdiv(csub(cc, root), cadd(cc, root));
        cd ec = cscale(eta, c);
        cd tm = cdiv(csub(ec, root), cadd(ec, root));
        double gk = kr * mt.rough_m * c;
        double rho = exp(-0.5 * gk * gk);
        b0 = cscale(cmul(te, b0), rho);
        b1 = cscale(cmul(tm, b1), rho);
        if (k + 1 < m) {
            const double* M = J + 4 + 4 * k;
            cd n0 = cadd(cscale(b0, M[0]), cscale(b1, M[1]));
            cd n1 = cadd(cscale(b0, M[2]), cscale(b1, M[3]));
            b0 = n0;
            b1 = n1;
        }
    }
    const double* cv = J + 32 + pb;
    cd proj = cadd(cscale(b0, cv[0]), cscale(b1, cv[1]));
    const double Lp = L[p];
    double amp = kC0 / (4.0 * kPi * f * Lp);
    double att = gamma ? exp10(-(double)gamma[fi] * Lp / 20000.0) : 1.0;
    double ph = disp ? -(double)disp[fi] * (kPi / 180.0) * Lp / 1000.0 : 0.0;
    double sn, cs;
    sincos(ph, &sn, &cs);
    cd v = cmul(cscale(cd{cs, sn}, amp * att), proj);
    g[t] = make_float2((float)v.re, (float)v.im);
}

}  // namespace

sbr_status gains_run(const sbr_path_list* pl, const sbr_material* mats, int32_t S,
                     const double* freqs, int32_t F, const float* gamma, const float* disp,
                     int32_t pol, float2* g, cudaStream_t s) {
    int64_t n = pl->P * (int64_t)F;
    if (n == 0) return SBR_OK;
    ::sbr::note_launch(), k_gains<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pl->P, F, pl->nb, pl->surf, pl->L, pl->jones,
                                                          mats, S, freqs, gamma, disp, pol, g);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

}  // namespace sbr
