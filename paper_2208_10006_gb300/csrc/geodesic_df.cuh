// Geodesic launch direction of ray `id` (Sec. II-A.1, Fig. 1) in double-float,
// computed where the ray is launched: no direction table is stored or read.
//
// The icosahedron's vertex coordinates are 0, +-1 and +-phi, i.e. A + B phi
// with integers A, B in {-1, 0, 1}. A class-I frequency-N lattice point is
//   P = (N - i - j) V_a + i V_b + j V_c    (N times the flat point),
// so each coordinate of P is exactly A + B phi with integers |A|, |B| <= N,
// and |P|^2 = C + D phi with C = sum(A^2 + B^2), D = sum(2 A B + B^2)
// (phi^2 = phi + 1), also exact integers. Only phi and the normalisation are
// rounded: the coordinates are formed in double-float from the integers, and
// 1 / sqrt(|P|^2) takes one Newton step in double-float from the FP32
// reciprocal square root, so the direction is accurate to ~1e-14, the
// accuracy of the double-float ray state that carries it.
//
// Ray ids follow the enumeration of the FP64 form (geodesic.cuh): 12 vertices,
// then N-1 points per sorted edge, then (N-1)(N-2)/2 interior points per
// sorted face, rows i = 1..N-2 (outer), columns j = 1..N-1-i.
#pragma once
#include "dfloat.cuh"
#include "sbr_internal.cuh"

namespace sbr {

struct IcoLattice {
    int8_t A[12][3], B[12][3];   // vertex coordinate = A + B phi
    int8_t e[30][2];             // sorted edges
    int8_t f[20][3];             // sorted faces
    float phi_hi, phi_lo;        // phi as double-float
};

IcoLattice make_ico_lattice();   // host: from make_ico()

// per-subdivision constants of the decode: the point counts of an edge (N-1)
// and of a face interior (N-1)(N-2)/2 with their FP32 reciprocals, which
// replace the integer divisions by a multiply and an exact correction
struct GeoN {
    int32_t N;
    uint32_t m;          // (N-1)(N-2)/2
    float inv_nm1, inv_m;
};

inline GeoN make_geo_n(int N) {
    GeoN g;
    g.N = N;
    g.m = (uint32_t)((int64_t)(N - 1) * (N - 2) / 2);
    g.inv_nm1 = N > 1 ? 1.0f / (float)(N - 1) : 0.f;
    g.inv_m = g.m > 0 ? 1.0f / (float)g.m : 0.f;
    return g;
}

// r / d for d >= 1 from an FP32 estimate of the quotient, corrected exactly
__device__ __forceinline__ uint32_t div_est(uint32_t r, uint32_t d, float inv) {
    uint32_t q = (uint32_t)fmaxf((float)r * inv, 0.f);
    while ((unsigned long long)q * d > r) --q;
    while ((unsigned long long)(q + 1) * d <= r) ++q;
    return q;
}

__device__ __forceinline__ df df_from_int(long long v) {
    const float h = (float)v;
    return df{h, (float)(v - (long long)h)};
}

// unit direction of the lattice point with integer coordinates A + B phi
__device__ __forceinline__ df3 lattice_unit_df(const IcoLattice& t, const int* PA, const int* PB) {
    long long C = 0, D = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        C += (long long)PA[k] * PA[k] + (long long)PB[k] * PB[k];
        D += 2LL * PA[k] * PB[k] + (long long)PB[k] * PB[k];
    }
    const df phi{t.phi_hi, t.phi_lo};
    // |P|^2 = C + D phi, then 1 / |P| from rsqrt and one Newton step:
    // y = y0 (1 + (1 - S y0^2) / 2)
    const df S = df_fma(df_from_int(C), df_from_int(D), phi);
    const float y0 = rsqrtf(S.hi);
    const df e = df_sub(df{1.f, 0.f}, df_mul(S, two_prod(y0, y0)));
    const df y = fast_two_sum(y0, __fmul_rn(__fmul_rn(y0, 0.5f), e.hi));
    df c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // A + B phi, exact products of the integers with phi's two words
        df x = two_prod((float)PB[k], t.phi_hi);
        x.lo = __fmaf_rn((float)PB[k], t.phi_lo, x.lo);
        x = df_add(df{(float)PA[k], 0.f}, x);
        c[k] = df_mul(x, y);
    }
    return df3{c[0], c[1], c[2]};
}

// lattice point (N - i - j) V_a + i V_b + j V_c of face f, as A + B phi
__device__ __forceinline__ void face_point(const IcoLattice& t, int f, int N, int i, int j, int* PA, int* PB) {
    const int va = t.f[f][0], vb = t.f[f][1], vc = t.f[f][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        PA[k] = (N - i - j) * t.A[va][k] + i * t.A[vb][k] + j * t.A[vc][k];
        PB[k] = (N - i - j) * t.B[va][k] + i * t.B[vb][k] + j * t.B[vc][k];
    }
}

__device__ __forceinline__ df3 geodesic_dir_df(const IcoLattice& t, const GeoN& g, uint32_t id) {
    const int N = g.N;
    int va, vb, vc, wa, wb, wc;
    if (id < 12u) {
        va = vb = vc = (int)id;
        wa = 1; wb = wc = 0;
    } else {
        uint32_t r = id - 12u;
        const uint32_t ne = 30u * (uint32_t)(N - 1);
        if (r < ne) {
            const uint32_t e = div_est(r, (uint32_t)(N - 1), g.inv_nm1);
            const int k = (int)(r - e * (uint32_t)(N - 1)) + 1;
            va = t.e[e][0]; vb = t.e[e][1]; vc = va;
            wa = N - k; wb = k; wc = 0;
        } else {
            r -= ne;
            const uint32_t m = g.m;
            const uint32_t f = div_est(r, m, g.inv_m);
            const int l = (int)(r - f * m);
            // row i holds N-1-i points; rows before i hold (i-1)(N-1) - i(i-1)/2:
            // the FP32 root of that quadratic, then exact integer corrections
            auto before = [N](int ii) { return (ii - 1) * (N - 1) - ii * (ii - 1) / 2; };
            const float b2 = 2.0f * (float)N - 1.0f;
            const float disc = fmaxf(b2 * b2 - 8.0f * (float)l - 8.0f * (float)(N - 1), 0.f);
            int i = (int)floorf(0.5f * (b2 - sqrtf(disc)));
            i = max(1, min(i, N - 2));
            while (i > 1 && before(i) > l) --i;
            while (i < N - 2 && before(i + 1) <= l) ++i;
            const int j = l - before(i) + 1;
            va = t.f[f][0]; vb = t.f[f][1]; vc = t.f[f][2];
            wa = N - i - j; wb = i; wc = j;
        }
    }
    int PA[3], PB[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        PA[k] = wa * t.A[va][k] + wb * t.A[vb][k] + wc * t.A[vc][k];
        PB[k] = wa * t.B[va][k] + wb * t.B[vb][k] + wc * t.B[vc][k];
    }
    return lattice_unit_df(t, PA, PB);
}

}  // namespace sbr
