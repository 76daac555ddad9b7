// Complex path gain g_n(f) of one path at one frequency (Eq. 1, 3, 6-10), FP64.
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
#pragma once
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
// a / b as a conj(b) / |b|^2: one FP64 division (FP64 is a narrow pipe on this
// GPU). The denominators here are cos + sqrt(eta - sin^2) and its TM form:
// |b|^2 stays far inside the FP64 range for any physical permittivity,
// conductivity and incidence angle.
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    const double inv = 1.0 / (b.re * b.re + b.im * b.im);
    return cd{(a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv};
}
// principal square root; the larger part is sqrt((|z| + |re|) / 2) and the
// other im / (2 that), so neither cancels
__device__ __forceinline__ cd csqrt_(cd z) {
    const double r = sqrt(z.re * z.re + z.im * z.im);
    if (r == 0.0) return cd{0.0, 0.0};
    const double u = sqrt(0.5 * (r + fabs(z.re)));
    const double v = 0.5 * fabs(z.im) / u;
    if (z.re >= 0.0) return cd{u, z.im < 0.0 ? -v : v};
    return cd{v, z.im < 0.0 ? -u : u};
}

// Fresnel coefficients (TE, TM) of reflection k and its roughness factor rho
// at frequency f; cosine of incidence c from the polarimetric record
struct Refl {
    cd te, tm;
    double rho;
};
__device__ __forceinline__ Refl reflection(const sbr_material& mt, double c, double f) {
    const double eps2_scale = 1.0 / (2.0 * kPi * f * kEps0);
    const double kr = 4.0 * kPi * f / kC0;
    double s2 = 1.0 - c * c;
    cd eta{mt.eps_r, -mt.sigma_s_per_m * eps2_scale};
    cd root = csqrt_(cd{eta.re - s2, eta.im});
    cd cc{c, 0.0};
    Refl r;
    r.te = cdiv(csub(cc, root), cadd(cc, root));
    cd ec = cscale(eta, c);
    r.tm = cdiv(csub(ec, root), cadd(ec, root));
    double gk = kr * mt.rough_m * c;
    r.rho = exp(-0.5 * gk * gk);
    return r;
}

// the field (b0, b1) through reflection k (coefficients rf), then the change to
// the next reflection's basis (k + 1 < m)
__device__ __forceinline__ void reflect_field(cd& b0, cd& b1, const Refl& rf, const double* __restrict__ J,
                                              int k, int m) {
    b0 = cscale(cmul(rf.te, b0), rf.rho);
    b1 = cscale(cmul(rf.tm, b1), rf.rho);
    if (k + 1 < m) {
        const double* M = J + 4 + 4 * k;
        cd n0 = cadd(cscale(b0, M[0]), cscale(b1, M[1]));
        cd n1 = cadd(cscale(b0, M[2]), cscale(b1, M[3]));
        b0 = n0;
        b1 = n1;
    }
}

// Rx projection, Friis amplitude, absorption and dispersion phase of the field
__device__ __forceinline__ float2 finish_gain(cd b0, cd b1, const double* __restrict__ J, int pb, double Lp,
                                              double f, const float* gamma, const float* disp) {
    const double* cv = J + 32 + pb;
    cd proj = cadd(cscale(b0, cv[0]), cscale(b1, cv[1]));
    double amp = kC0 / (4.0 * kPi * f * Lp);
    double att = gamma ? exp10(-(double)*gamma * Lp / 20000.0) : 1.0;
    double ph = disp ? -(double)*disp * (kPi / 180.0) * Lp / 1000.0 : 0.0;
    double sn, cs;
    sincos(ph, &sn, &cs);
    cd v = cmul(cscale(cd{cs, sn}, amp * att), proj);
    return make_float2((float)v.re, (float)v.im);
}

// m reflections off surfaces surf[0..m), unfolded length Lp, polarimetric
// record J (kJones doubles); gamma / disp may be null (no absorption / phase)
__device__ __forceinline__ float2 path_gain(int m, const int32_t* __restrict__ surf, double Lp,
                                            const double* __restrict__ J, const sbr_material* __restrict__ mats,
                                            int32_t S, double f, const float* gamma, const float* disp, int pol) {
    const int pb = pol == SBR_POL_V ? 0 : 2;
    cd b0{J[pb], 0.0}, b1{J[pb + 1], 0.0};
    for (int k = 0; k < m; ++k) {
        int s = surf[k];
        if (s < 0 || s >= S) return make_float2(NAN, NAN);  // not reachable: S is checked on the host
        reflect_field(b0, b1, reflection(mats[s], J[36 + k], f), J, k, m);
    }
    return finish_gain(b0, b1, J, pb, Lp, f, gamma, disp);
}

}  // namespace
}  // namespace sbr
