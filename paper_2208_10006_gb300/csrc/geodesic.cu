// Geodesic ray launching (Sec. II-A.1, Fig. 1): icosahedron tables (FP64
// and the exact integer lattice form the trace kernels decode), the direction
// list, and alpha, the largest angle between directions joined by
// a sub-triangle edge, which sizes the reception sphere (Sec. II-A.3).
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>

#include "dfloat.cuh"
#include "geodesic.cuh"
#include "geodesic_df.cuh"

namespace sbr {

// Icosahedron with vertices (0,+-1,+-phi), (+-1,+-phi,0), (+-phi,0,+-1), signs
// in the order (+,+), (+,-), (-,+), (-,-); edges are the vertex pairs at
// distance 2 and faces the mutually adjacent triples, both in lexicographic
// order of vertex index.
Ico make_ico() {
    Ico ico{};
    const double ph = (1.0 + std::sqrt(5.0)) / 2.0;
    const int sg[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
    for (int k = 0; k < 4; ++k) {
        double a = sg[k][0], b = sg[k][1];
        double* v0 = ico.v[k];
        v0[0] = 0; v0[1] = a; v0[2] = b * ph;
        double* v1 = ico.v[4 + k];
        v1[0] = a; v1[1] = b * ph; v1[2] = 0;
        double* v2 = ico.v[8 + k];
        v2[0] = a * ph; v2[1] = 0; v2[2] = b;
    }
    auto adjacent = [&](int a, int b) {
        double s = 0;
        for (int c = 0; c < 3; ++c) s += (ico.v[a][c] - ico.v[b][c]) * (ico.v[a][c] - ico.v[b][c]);
        return std::fabs(s - 4.0) < 1e-9;
    };
    int ne = 0, nf = 0;
    for (int a = 0; a < 12; ++a)
        for (int b = a + 1; b < 12; ++b)
            if (adjacent(a, b)) { ico.e[ne][0] = (int8_t)a; ico.e[ne][1] = (int8_t)b; ++ne; }
    for (int a = 0; a < 12; ++a)
        for (int b = a + 1; b < 12; ++b)
            for (int c = b + 1; c < 12; ++c)
                if (adjacent(a, b) && adjacent(b, c) && adjacent(a, c)) {
                    ico.f[nf][0] = (int8_t)a; ico.f[nf][1] = (int8_t)b; ico.f[nf][2] = (int8_t)c;
                    ++nf;
                }
    return ico;
}

namespace {

__global__ void k_dirs(const __grid_constant__ Ico ico, int N, int64_t R, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    d3 d = geodesic_dir(ico, N, (uint32_t)i);
    out[3 * i] = d.x; out[3 * i + 1] = d.y; out[3 * i + 2] = d.z;
}

__device__ __forceinline__ double angle_between(d3 a, d3 b) {
    return atan2(norm(cross(a, b)), dot(a, b));
}

// one thread per lattice point (face f, i, j) with i + j < N: the three
// edges of the upward sub-triangle (i,j)-(i+1,j)-(i,j+1) cover every
// sub-triangle edge of the face
__global__ void k_alpha(const __grid_constant__ Ico ico, int N, int64_t per_face,
                        unsigned long long* __restrict__ best) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (t < 20 * per_face) {
        int f = (int)(t / per_face);
        int64_t l = t % per_face;
        // row i has N - i points (j = 0..N-1-i); rows before i hold i(2N+1-i)/2
        auto before = [N](int64_t ii) { return ii * (2 * (int64_t)N + 1 - ii) / 2; };
        double b2 = 2.0 * N + 1.0;
        int64_t i = (int64_t)floor((b2 - sqrt(fmax(b2 * b2 - 8.0 * (double)l, 0.0))) / 2.0);
        if (i < 0) i = 0;
        while (i > 0 && before(i) > l) --i;
        while (i < N - 1 && before(i + 1) <= l) ++i;
        int64_t j = l - before(i);
        d3 a = ld3(ico.v[ico.f[f][0]]), b = ld3(ico.v[ico.f[f][1]]), c = ld3(ico.v[ico.f[f][2]]);
        d3 p00 = unit(a + ((b - a) * ((double)i / N) + (c - a) * ((double)j / N)));
        d3 p10 = unit(a + ((b - a) * ((double)(i + 1) / N) + (c - a) * ((double)j / N)));
        d3 p01 = unit(a + ((b - a) * ((double)i / N) + (c - a) * ((double)(j + 1) / N)));
        m = fmax(angle_between(p00, p10), fmax(angle_between(p00, p01), angle_between(p10, p01)));
    }
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(best, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_alpha_store(const unsigned long long* best, double* alpha) {
    *alpha = __longlong_as_double((long long)*best);
}

}  // namespace

IcoLattice make_ico_lattice() {
    const Ico ico = make_ico();
    const double ph = (1.0 + std::sqrt(5.0)) / 2.0;
    IcoLattice t{};
    for (int v = 0; v < 12; ++v)
        for (int k = 0; k < 3; ++k) {
            const double x = ico.v[v][k];
            const bool is_phi = std::fabs(std::fabs(x) - ph) < 1e-9;
            const int sg = x > 0 ? 1 : (x < 0 ? -1 : 0);
            t.A[v][k] = (int8_t)(is_phi ? 0 : sg);
            t.B[v][k] = (int8_t)(is_phi ? sg : 0);
        }
    for (int e = 0; e < 30; ++e)
        for (int k = 0; k < 2; ++k) t.e[e][k] = ico.e[e][k];
    for (int f = 0; f < 20; ++f)
        for (int k = 0; k < 3; ++k) t.f[f][k] = ico.f[f][k];
    const df p = df_from_double(ph);
    t.phi_hi = p.hi;
    t.phi_lo = p.lo;
    return t;
}

namespace {
// the double-float directions the trace kernels launch, widened to FP64
__global__ void k_dirs_df(const __grid_constant__ IcoLattice t, GeoN g, int64_t R, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    const df3 d = geodesic_dir_df(t, g, (uint32_t)i);
    out[3 * i] = df_to_double(d.x); out[3 * i + 1] = df_to_double(d.y); out[3 * i + 2] = df_to_double(d.z);
}
}  // namespace

namespace {
// squared chord |u - v|^2 of two unit directions in double-float (no
// cancellation: the differences of the components are formed first)
__device__ __forceinline__ df chord2(const df3& u, const df3& v) {
    const df x = df_sub(u.x, v.x), y = df_sub(u.y, v.y), z = df_sub(u.z, v.z);
    return df_fma(df_fma(df_mul(x, x), y, y), z, z);
}

// the larger of two double-float values (their hi words first, then lo)
__device__ __forceinline__ df df_max(df a, df b) { return (b.hi > a.hi || (b.hi == a.hi && b.lo > a.lo)) ? b : a; }

// alpha over the sub-triangle edges of one face: every face is the image of
// face 0 under a rotation of the icosahedron (an isometry that maps the
// lattice of one face onto that of another), so the largest edge angle is the
// same on all 20. One thread per upward sub-triangle (i, j) - (i+1, j) -
// (i, j+1), i + j <= N-1, whose three edges cover every edge of the face; the
// largest squared chord is reduced in double-float and stored as FP64 bits (a
// monotone order for non-negative values), and alpha = 2 asin(chord / 2)
// follows in FP64 once.
__global__ void k_alpha_df(const __grid_constant__ IcoLattice t, int N, int64_t per_face,
                           unsigned long long* __restrict__ best) {
    ::sbr::pdl_wait();
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    df m{0.f, 0.f};
    if (l < per_face) {
        // row i holds N - i points (j = 0..N-1-i); rows before i hold i(2N+1-i)/2
        auto before = [N](int64_t ii) { return ii * (2 * (int64_t)N + 1 - ii) / 2; };
        const float b2 = 2.0f * (float)N + 1.0f;
        int64_t i = (int64_t)floorf(0.5f * (b2 - sqrtf(fmaxf(b2 * b2 - 8.0f * (float)l, 0.f))));
        i = i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
        while (i > 0 && before(i) > l) --i;
        while (i < N - 1 && before(i + 1) <= l) ++i;
        const int j = (int)(l - before(i));
        int PA[3], PB[3];
        face_point(t, 0, N, (int)i, j, PA, PB);
        const df3 p00 = lattice_unit_df(t, PA, PB);
        face_point(t, 0, N, (int)i + 1, j, PA, PB);
        const df3 p10 = lattice_unit_df(t, PA, PB);
        face_point(t, 0, N, (int)i, j + 1, PA, PB);
        const df3 p01 = lattice_unit_df(t, PA, PB);
        m = df_max(chord2(p00, p10), df_max(chord2(p00, p01), chord2(p10, p01)));
    }
    for (int o = 16; o; o >>= 1) {
        const df b{__shfl_xor_sync(0xffffffffu, m.hi, o), __shfl_xor_sync(0xffffffffu, m.lo, o)};
        m = df_max(m, b);
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, (unsigned long long)__double_as_longlong(df_to_double(m)));
}

__global__ void k_alpha_df_store(const unsigned long long* best, double* alpha) {
    ::sbr::pdl_wait();
    const double c2 = __longlong_as_double((long long)*best);
    *alpha = 2.0 * asin(0.5 * sqrt(c2));
}
}  // namespace

sbr_status launch_alpha_fast(int32_t N, double* alpha, cudaStream_t s) {
    const int64_t per_face = (int64_t)N * (N + 1) / 2;
    unsigned long long* best;
    SBR_TRY(dalloc_n(&best, 1, s));
    SBR_TRY_CUDA(cudaMemsetAsync(best, 0, sizeof(unsigned long long), s));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_alpha_df, dim3((unsigned)((per_face + 255) / 256)), dim3(256), 0, s, make_ico_lattice(), N,
                                                                                          per_face, best);
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_alpha_df_store, dim3(1), dim3(1), 0, s, best, alpha);
    SBR_TRY_CUDA(cudaGetLastError());
    dfree(best, s);
    return SBR_OK;
}

sbr_status launch_dirs(int32_t N, double* dirs, cudaStream_t s) {
    int64_t R = 10 * (int64_t)N * N + 2;
    // test hook: SBR_DIRS_DF=1 returns the double-float directions the trace
    // kernels compute where they launch a ray (instead of the FP64 form)
    const char* e = getenv("SBR_DIRS_DF");
    if (e && e[0] == '1') {
        ::sbr::note_launch(), k_dirs_df<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(make_ico_lattice(), make_geo_n(N), R,
                                                                                 dirs);
    } else {
        Ico ico = make_ico();
        ::sbr::note_launch(), k_dirs<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(ico, N, R, dirs);
    }
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

sbr_status launch_alpha(int32_t N, double* alpha, cudaStream_t s) {
    Ico ico = make_ico();
    int64_t per_face = (int64_t)N * (N + 1) / 2;
    unsigned long long* best;
    SBR_TRY(dalloc_n(&best, 1, s));
    SBR_TRY_CUDA(cudaMemsetAsync(best, 0, sizeof(unsigned long long), s));
    int64_t tot = 20 * per_face;
    ::sbr::note_launch(), k_alpha<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ico, N, per_face, best);
    ::sbr::note_launch(), k_alpha_store<<<1, 1, 0, s>>>(best, alpha);
    SBR_TRY_CUDA(cudaGetLastError());
    dfree(best, s);
    return SBR_OK;
}

}  // namespace sbr
