// Shoot and bounce (Sec. II-A.2 ray tracing, Sec. II-A.3 reception), run
// breadth-first as in Sec. I ("width first search"): one persistent launch
// per bounce over a compacted queue of live rays.
//
// Per segment:
//  1. closest hit by FP32 BVH traversal with the watertight ray/triangle test
//     of Woop, Benthin and Wald (JCGT 2013). The traversal also records how
//     close the decision was: the barycentric margin of the hit, near misses
//     of faces in front, hits of other surfaces within a relative margin of
//     t, and grazing incidence.
//  2. a decision closer than kCert (relative) to any of those boundaries is
//     re-made by an FP64 traversal that applies the exact rule of the
//     specification (smallest t > 0, ties to the lower face id, every face of
//     the surface reflected last ignored). Otherwise the FP32 face stands and
//     only its t is recomputed in FP64 from the face plane.
//  3. reception: receivers near the segment are found through a BVH over the
//     receiver points (boxes grown by the largest sphere radius on the
//     segment); each is tested exactly in FP64: t* = (Rx-o).d in [0, t_hit]
//     and |o + t* d - Rx| <= alpha (L + t*) / sqrt(3).
//  4. received (rx, surface sequence) keys go into a device hash table that
//     keeps min(dist, ray id) per key with a 64-bit atomicMin.
//  5. specular bounce d' = d - 2 (d.n) n in FP64, unfolded length L += t,
//     survivors appended to the next queue with one atomic per warp.
// The ray state (origin, direction, unfolded length L) is kept in double-FP32
// (about 48 significant bits), so that the hit and reception decisions agree
// with an FP64 evaluation of the same rule to rounding while the arithmetic
// stays on the FP32 pipes (FP64 throughput on this GPU is a small fraction of
// FP32). FP64 is used only to re-decide uncertain faces exactly. The FP32
// traversal runs on the high words and carries the per-triangle cost.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "batch.cuh"
#include "dfloat.cuh"
#include "geodesic.cuh"
#include "geodesic_df.cuh"

namespace sbr {
namespace {

constexpr int kStack = 64;
constexpr int kTraceThreads = 128;
constexpr int kSpinLimit = 1 << 20;    // bounded wait for a dedup slot being published

struct RayRec {
    float oh[3], ol[3];  // origin, double-float
    float dh[3], dl[3];  // direction, double-float
    float Lh, Ll;        // unfolded length, double-float
    uint32_t ray;
    int32_t prev;
};
static_assert(sizeof(RayRec) == 64, "ray record is one 64-byte line");

struct TraceArgs {
    const float4* nodes;
    const float4* tris;      // [T*3] BVH-order faces, the last of three axis-rotated copies
    const float4* plane;     // [T*2] double-float face planes, BVH order
    int64_t T;
    int64_t rot_stride;      // 3 T: float4s between the rotated copies
    const float4* rx_nodes;
    const int32_t* rx_order;
    const float4* rx_df;     // [n_rx*2] receiver positions, double-float
    const float* rx_root;
    int32_t n_rx;
    const float4* alpha_df;  // (alpha hi, lo, alpha^2/3 hi, lo)
    IcoLattice ico;          // launch grid: directions decoded per ray in double-float
    GeoN geo;                // its subdivision constants
    int N, K, bounce;
    int64_t R;               // rays of the launch grid
    int64_t ray0, Rr;        // the traced id range [ray0, ray0 + Rr) (the whole grid by default)
    // launch order of the rays: the vertex and edge rays first, then the 20
    // faces' interior rays face by face in the order face_order (their ids
    // stay the geodesic ids)
    int64_t pool_pre, pool_face;
    uint8_t face_order[20];
    float tx_h[3], tx_l[3];
    const RayRec* qin;
    RayRec* qout;
    const unsigned long long* n_in;
    unsigned long long* n_out;
    unsigned long long* work;
    int32_t* seq;
    int32_t* seqf;           // [K][R] face hit at each bounce (refinement hints)
    uint32_t* ht_state;
    uint32_t* ht_key;
    unsigned long long* ht_val;
    uint32_t ht_mask;
    TraceCountersDev* cnt;
};

// geodesic id of the i-th ray launched (a range trace launches its ids in order)
__device__ __forceinline__ uint32_t pool_ray(const TraceArgs& a, unsigned long long i) {
    const int64_t r = (int64_t)i - a.pool_pre;
    if (r < 0 || a.pool_face == 0) return (uint32_t)(a.ray0 + (int64_t)i);
    const int64_t k = r / a.pool_face;
    return (uint32_t)(a.pool_pre + (int64_t)a.face_order[k] * a.pool_face + (r - k * a.pool_face));
}

__device__ __forceinline__ float comp3(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// The FP32 ray of the watertight test. kz is the dominant axis of the
// direction, kx = kz + 1 and ky = kz + 2 (mod 3) follow it cyclically: the test
// is two-sided (the sign of det absorbs the orientation), so the axes are not
// swapped for a negative dz, and the faces are read from the copy whose vertex
// components are stored in this (kx, ky, kz) order.
struct Ray32 {
    float3 ok;         // origin in the shear frame's axis order (kx, ky, kz)
    float3 inv, oinv;  // oinv = o * inv, for the slab test fma(lo, inv, -oinv)
    int kz;
    float Sx, Sy, Sz;
};

// reciprocal of a direction component for the slab tests; an exact zero
// becomes +-2^-80 so that inv and o * inv stay finite. The fast division (a
// few ulp for |x| in [2^-80, 1]) suffices: the slab tests only cull, and their
// rounding stays far inside the boxes' relative padding (2^-20 of |x| + 1 in
// the scene tree, the sphere radius and 1e-5 of the coordinates in the
// receiver tree)
__device__ __forceinline__ float safe_rcp(float x) {
    const float tiny = 8.271806e-25f;  // 2^-80
    return __fdividef(1.0f, fabsf(x) > tiny ? x : copysignf(tiny, x));
}

__device__ __forceinline__ Ray32 make_ray32(float3 o, float3 d) {
    Ray32 r;
    r.inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    r.oinv = make_float3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    r.kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    const int kx = r.kz == 2 ? 0 : r.kz + 1, ky = kx == 2 ? 0 : kx + 1;
    float dz = comp3(d, r.kz);
    r.Sx = comp3(d, kx) / dz;
    r.Sy = comp3(d, ky) / dz;
    r.ok = make_float3(comp3(o, kx), comp3(o, ky), comp3(o, r.kz));
    r.Sz = 1.0f / dz;
    return r;
}

// slab test, t = lo / d - o / d as one fma per plane; its rounding (~eps |o|
// in distance) is far inside the relative padding of the BVH boxes
__device__ __forceinline__ bool box_hit(float lx, float ly, float lz, float hx, float hy, float hz,
                                        const Ray32& r, float tmax, float& tnear) {
    float t0x = fmaf(lx, r.inv.x, -r.oinv.x), t1x = fmaf(hx, r.inv.x, -r.oinv.x);
    float t0y = fmaf(ly, r.inv.y, -r.oinv.y), t1y = fmaf(hy, r.inv.y, -r.oinv.y);
    float t0z = fmaf(lz, r.inv.z, -r.oinv.z), t1z = fmaf(hz, r.inv.z, -r.oinv.z);
    float tmin = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.f));
    float tmx = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    tnear = tmin;
    return tmin <= tmx;
}

// Certification of the FP32 decisions. For every tested face the edge
// functions U, V, W of the watertight test carry a rounding-error bound
//   errE = 8 eps max(|Cx By| + |Cy Bx|, |Ax Cy| + |Ay Cx|, |Bx Ay| + |By Ax|)
//        + 4 eps (|o|_inf + t_scale) (perimeter of the sheared triangle)
// (eps = 2^-24): the first term covers the arithmetic of the test, the second
// the rounding of the double-float ray to FP32. It is evaluated through the
// upper bound 8 eps (Sx Sy + (|o|_inf + t_scale)(Sx + Sy)). A face is a certain miss if some edge
// function is below -errE, a certain hit if all exceed +errE and t is clearly
// positive. Everything in between, and hits of different surfaces whose t
// agree within kTie, go to a short list that is re-decided in FP64 with the
// exact rule; only a full list falls back to a complete FP64 traversal.
constexpr int kUnc = 6;
constexpr float kEps32 = 5.9604645e-8f;
constexpr float kTie = 1e-5f;

struct Trav {
    float best_t, lim, omax;
    int32_t best_j, best_face, best_surf;
    int nu;
    bool overflow;
    int32_t unc[kUnc];
};

__device__ __forceinline__ void push_unc(Trav& tv, int32_t j) {
    for (int k = 0; k < tv.nu; ++k)
        if (tv.unc[k] == j) return;
    if (tv.nu < kUnc) tv.unc[tv.nu++] = j;
    else tv.overflow = true;
}

__device__ __forceinline__ void tri_test32(const float4* __restrict__ tris, int32_t j, int prev,
                                           const Ray32& r, Trav& tv) {
    float4 a = __ldg(tris + 3 * j), b = __ldg(tris + 3 * j + 1), c = __ldg(tris + 3 * j + 2);
    int32_t surf = __float_as_int(a.w);
    if (surf == prev) return;
    float Ax = a.x - r.ok.x, Ay = a.y - r.ok.y, Az = a.z - r.ok.z;
    float Bx = b.x - r.ok.x, By = b.y - r.ok.y, Bz = b.z - r.ok.z;
    float Cx = c.x - r.ok.x, Cy = c.y - r.ok.y, Cz = c.z - r.ok.z;
    Ax = fmaf(-r.Sx, Az, Ax); Ay = fmaf(-r.Sy, Az, Ay);
    Bx = fmaf(-r.Sx, Bz, Bx); By = fmaf(-r.Sy, Bz, By);
    Cx = fmaf(-r.Sx, Cz, Cx); Cy = fmaf(-r.Sy, Cz, Cy);
    float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
    float det = U + V + W;
    float sg = det >= 0.f ? 1.f : -1.f;
    float mn = fminf(fminf(sg * U, sg * V), sg * W);  // min of the orientation-adjusted values
    // bound of the rounding error of U, V, W (see above), in a cheaper looser form:
    // each |Cx By| + |Cy Bx| <= Sx Sy and the sheared perimeter <= 2 (Sx + Sy)
    float Sx = fabsf(Ax) + fabsf(Bx) + fabsf(Cx), Sy = fabsf(Ay) + fabsf(By) + fabsf(Cy);
    float zs = fmaxf(fabsf(Az), fmaxf(fabsf(Bz), fabsf(Cz)));
    float errE = 8.f * kEps32 * fmaf(Sx, Sy, (tv.omax + zs) * (Sx + Sy));
    if (mn < -errE) return;  // certainly outside one edge
    float adet = fabsf(det);
    if (!(adet > 3.f * errE)) {  // t is not reliable: let FP64 decide
        push_unc(tv, j);
        return;
    }
    Az *= r.Sz; Bz *= r.Sz; Cz *= r.Sz;
    float t = (U * Az + V * Bz + W * Cz) / det;
    float tiny = 1e-5f * (tv.omax + 1.f);
    if (t < -tiny || t > tv.lim) return;
    if (mn > errE && t > tiny) {
        int face = __float_as_int(b.w);
        float tol = kTie * fmaxf(t, tv.best_t) + 16.f * kEps32 * (tv.omax + fmaxf(t, tv.best_t));
        if (tv.best_j >= 0 && surf != tv.best_surf && fabsf(t - tv.best_t) <= tol) {
            push_unc(tv, j);
            push_unc(tv, tv.best_j);
        }
        if (t < tv.best_t || (t == tv.best_t && face < tv.best_face)) {
            tv.best_t = t; tv.best_j = j; tv.best_face = face; tv.best_surf = surf;
            tv.lim = t * (1.f + 4.f * kTie) + tiny;
        }
    } else {
        push_unc(tv, j);
    }
}

// FP32 closest hit. Returns the sorted triangle index of the certain best
// (or -1) and the list of faces that FP64 must re-decide. kCount adds node
// visits and triangle tests to *visits / *tests (instrumented traces).
// A is the kernel's argument block (or a per-job view of it) with the scene
// fields nodes, tris and the counters cnt.
template <bool kCount, class A>
__device__ int32_t traverse32(const A& a, const Ray32& r, int prev, Trav& tv, int* stack,
                              unsigned* visits, unsigned* tests) {
    tv.best_t = INFINITY; tv.lim = INFINITY; tv.best_j = -1; tv.best_face = 0x7fffffff;
    tv.best_surf = -2; tv.nu = 0; tv.overflow = false;
    tv.omax = fmaxf(fabsf(r.ok.x), fmaxf(fabsf(r.ok.y), fabsf(r.ok.z)));
    // while-while: the inner loop descends through internal nodes (each tests
    // its two child boxes and continues with the nearer hit child, the farther
    // one stacked) until it reaches a leaf reference, whose triangles the
    // outer loop then tests; leaves and nodes share the stack. The faces are
    // read with vertex components in this ray's (kx, ky, kz) order: block kz of
    // the three rotated copies, of which a.tris is the last
    const float4* tris_k = a.tris + (int64_t)(r.kz - 2) * a.rot_stride;
    int sp = 0;
    int32_t ref = 0;
    for (;;) {
        while (ref >= 0) {
            const float4* nd = a.nodes + 4 * (int64_t)ref;
            float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            int32_t r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
            if (kCount) ++*visits;
            float tn0, tn1;
            bool h0 = box_hit(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, r, tv.lim, tn0);
            bool h1 = box_hit(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, r, tv.lim, tn1);
            const bool first0 = h0 && (!h1 || tn0 <= tn1);
            if (h0 && h1) {
                if (sp == kStack) { atomicOr(&a.cnt->status, (unsigned)ST_STACK); tv.overflow = true; return tv.best_j; }
                stack[sp++] = first0 ? r1 : r0;
            }
            if (h0 || h1) ref = first0 ? r0 : r1;
            else if (sp == 0) return tv.best_j;
            else ref = stack[--sp];
        }
        const int32_t first = leaf_first(ref), cnt = leaf_count(ref);
        for (int k = 0; k < cnt; ++k) tri_test32(tris_k, first + k, prev, r, tv);
        if (kCount) *tests += cnt;
        if (sp == 0) break;
        ref = stack[--sp];
    }
    return tv.best_j;
}

// FP64 Moller-Trumbore: the exact rule, used when FP32 is not conclusive
__device__ __forceinline__ bool mt64(const float4* __restrict__ tris, int32_t j, d3 o, d3 d,
                                     double& t) {
    float4 a = __ldg(tris + 3 * j), b = __ldg(tris + 3 * j + 1), c = __ldg(tris + 3 * j + 2);
    d3 v0 = mk3(a.x, a.y, a.z), v1 = mk3(b.x, b.y, b.z), v2 = mk3(c.x, c.y, c.z);
    d3 e1 = v1 - v0, e2 = v2 - v0;
    d3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return false;
    double inv = 1.0 / det;
    d3 s = o - v0;
    double u = dot(s, p) * inv;
    d3 q = cross(s, e1);
    double v = dot(d, q) * inv;
    t = dot(e2, q) * inv;
    return u >= 0.0 && v >= 0.0 && (1.0 - u - v) >= 0.0 && t > 0.0;
}

// smallest FP64 barycentric of the segment's hit on face j (instrumented
// traces: a hit at or below 1e-6 is edge-ambiguous in the parity rule)
__device__ __forceinline__ double min_bary64(const float4* __restrict__ tris, int32_t j, d3 o, d3 d) {
    float4 a = __ldg(tris + 3 * j), b = __ldg(tris + 3 * j + 1), c = __ldg(tris + 3 * j + 2);
    d3 v0 = mk3(a.x, a.y, a.z), v1 = mk3(b.x, b.y, b.z), v2 = mk3(c.x, c.y, c.z);
    d3 e1 = v1 - v0, e2 = v2 - v0;
    d3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return 0.0;
    double inv = 1.0 / det;
    d3 s = o - v0;
    double u = dot(s, p) * inv;
    double v = dot(d, cross(s, e1)) * inv;
    return fmin(fmin(u, v), 1.0 - u - v);
}

__device__ __forceinline__ bool box_hit64(const float* b, d3 o, d3 inv, double tmax) {
    double t0x = ((double)b[0] - o.x) * inv.x, t1x = ((double)b[3] - o.x) * inv.x;
    double t0y = ((double)b[1] - o.y) * inv.y, t1y = ((double)b[4] - o.y) * inv.y;
    double t0z = ((double)b[2] - o.z) * inv.z, t1z = ((double)b[5] - o.z) * inv.z;
    double tmin = fmax(fmax(fmin(t0x, t1x), fmin(t0y, t1y)), fmax(fmin(t0z, t1z), 0.0));
    double tmx = fmin(fmin(fmax(t0x, t1x), fmax(t0y, t1y)), fmin(fmax(t0z, t1z), tmax));
    return tmin <= tmx;
}

template <class A>
__device__ __noinline__ int32_t traverse64(const A& a, d3 o, d3 d, int prev, double& t_out, int* stack) {
    d3 inv = mk3(1.0 / d.x, 1.0 / d.y, 1.0 / d.z);
    double best_t = INFINITY;
    int32_t best_j = -1, best_face = 0x7fffffff;
    int sp = 0;
    int32_t node = 0;
    for (;;) {
        const float4* nd = a.nodes + 4 * (int64_t)node;
        float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        float b0[6] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y};
        float b1[6] = {n1.z, n1.w, n2.x, n2.y, n2.z, n2.w};
        int32_t r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
        double lim = best_t * (1.0 + 1e-12);
        bool h0 = box_hit64(b0, o, inv, lim);
        bool h1 = box_hit64(b1, o, inv, lim) && r1 != r0;
        for (int c = 0; c < 2; ++c) {
            int32_t rr = c ? r1 : r0;
            bool hh = c ? h1 : h0;
            if (hh && rr < 0) {
                const int32_t first = leaf_first(rr), cnt = leaf_count(rr);
                for (int32_t j = first; j < first + cnt; ++j) {
                    float4 a0 = __ldg(a.tris + 3 * j), a1 = __ldg(a.tris + 3 * j + 1);
                    if (__float_as_int(a0.w) == prev) continue;
                    double t;
                    int face = __float_as_int(a1.w);
                    if (mt64(a.tris, j, o, d, t) && (t < best_t || (t == best_t && face < best_face))) {
                        best_t = t; best_j = j; best_face = face;
                    }
                }
                if (c) h1 = false; else h0 = false;
            }
        }
        if (h0 && h1) {
            if (sp < kStack) stack[sp++] = r1;
            else { atomicOr(&a.cnt->status, (unsigned)ST_STACK); break; }
            node = r0;
        } else if (h0) {
            node = r0;
        } else if (h1) {
            node = r1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    t_out = best_t;
    return best_j;
}

// ---------------------------------------------------------------- dedup table
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85ebca6bu; h ^= h >> 13; h *= 0xc2b2ae35u; h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint32_t key_hash(const uint32_t* key) {
    uint32_t h = 0x9747b28cu;
    for (int k = 0; k < kKeyWords; ++k) h = mix32(h ^ (key[k] + 0x9e3779b9u + (h << 6) + (h >> 2)));
    return h;
}

template <class A>
__device__ void ht_insert(const A& a, const uint32_t* key, unsigned long long val) {
    uint32_t h = key_hash(key) & a.ht_mask;
    for (uint32_t probe = 0; probe <= a.ht_mask; ++probe) {
        uint32_t s = (h + probe) & a.ht_mask;
        uint32_t st = atomicCAS(&a.ht_state[s], 0u, 1u);
        if (st == 0u) {
            for (int k = 0; k < kKeyWords; ++k) a.ht_key[(size_t)s * kKeyWords + k] = key[k];
            __threadfence();
            atomicExch(&a.ht_state[s], 2u);
            atomicMin(&a.ht_val[s], val);
            atomicAdd(&a.cnt->keys, 1ull);
            return;
        }
        int spins = 0;
        while (*((volatile uint32_t*)&a.ht_state[s]) != 2u) {
            if (++spins > kSpinLimit) {
                atomicOr(&a.cnt->status, (unsigned)ST_TIMEOUT);
                return;
            }
            __nanosleep(32);
        }
        __threadfence();
        bool eq = true;
        const volatile uint32_t* kk = a.ht_key + (size_t)s * kKeyWords;
        for (int k = 0; k < kKeyWords; ++k) eq = eq && (kk[k] == key[k]);
        if (eq) {
            atomicMin(&a.ht_val[s], val);
            return;
        }
    }
    atomicOr(&a.cnt->status, (unsigned)ST_CAPACITY);
}

// ---------------------------------------------------------------- reception
// exact double-float test of one receiver R against the segment [0, t_hit]
// (or the open ray when there is no hit); dist = closest-approach distance
__device__ __forceinline__ bool rx_accept(const df3& o, const df3& d, df L, df t_hit, bool hit,
                                          const df3& R, df a2o3, float& dist) {
    df3 v = df3_sub(R, o);
    df ts = df3_dot(v, d);
    if (ts.hi < 0.f || (hit && df_lt(t_hit, ts))) return false;
    df3 w = df3_fma(df3{df_neg(v.x), df_neg(v.y), df_neg(v.z)}, d, ts);   // o + t* d - Rx
    df dist2 = df3_dot(w, w);
    df sl = df_add(L, ts);
    df rad2 = df_mul(a2o3, df_mul(sl, sl));
    if (!df_le(dist2, rad2) || (ts.hi == 0.f && ts.lo < 0.f)) return false;
    dist = sqrtf(fmaxf(dist2.hi, 0.f));
    return true;
}

// Receivers near the segment come from a BVH over the receiver points whose
// boxes are grown by the largest sphere radius on the segment (FP32,
// conservative); each is then tested exactly in double-float:
//   t* = (Rx - o).d in [0, t_hit],  |o + t* d - Rx|^2 <= alpha^2 (L + t*)^2 / 3.
template <bool kCount>
__device__ void receive(const TraceArgs& a, int bounce, const df3& o, const df3& d, df L, df t_hit, bool hit,
                        const Ray32& r, uint32_t ray, int* stack, unsigned* rx_visits) {
    if (a.n_rx <= 0) return;
    const float4 al = __ldg(a.alpha_df);
    const df a2o3 = df_make(al.z, al.w);
    float t_end = t_hit.hi;
    if (!hit) {
        // no receiver lies farther than the centre of their box plus its half diagonal
        float cx = 0.5f * (a.rx_root[0] + a.rx_root[3]) - o.x.hi;
        float cy = 0.5f * (a.rx_root[1] + a.rx_root[4]) - o.y.hi;
        float cz = 0.5f * (a.rx_root[2] + a.rx_root[5]) - o.z.hi;
        float hx = a.rx_root[3] - a.rx_root[0], hy = a.rx_root[4] - a.rx_root[1], hz = a.rx_root[5] - a.rx_root[2];
        t_end = (sqrtf(cx * cx + cy * cy + cz * cz) + 0.5f * sqrtf(hx * hx + hy * hy + hz * hz)) * (1.f + 1e-5f) + 1e-3f;
    }
    float rmax = al.x * (L.hi + t_end) * 0.57735027f * (1.f + 1e-4f) +
                 1e-5f * (fabsf(o.x.hi) + fabsf(o.y.hi) + fabsf(o.z.hi) + L.hi + t_end);
    float tmax = t_end * (1.f + 1e-5f) + rmax;
    // the segment against the receivers' (padded) root box grown by rmax: it
    // contains every grown child box, so a miss here is a miss of the whole
    // tree, and most segments pass far from every receiver
    {
        float tn;
        if (!box_hit(a.rx_root[0] - rmax, a.rx_root[1] - rmax, a.rx_root[2] - rmax, a.rx_root[3] + rmax,
                     a.rx_root[4] + rmax, a.rx_root[5] + rmax, r, tmax, tn))
            return;
    }
    int sp = 0;
    int32_t node = 0;
    for (;;) {
        const float4* nd = a.rx_nodes + 4 * (int64_t)node;
        float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        int32_t r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
        if (kCount) ++*rx_visits;
        float tn0, tn1;
        bool h0 = box_hit(n0.x - rmax, n0.y - rmax, n0.z - rmax, n0.w + rmax, n1.x + rmax, n1.y + rmax,
                          r, tmax, tn0);
        bool h1 = box_hit(n1.z - rmax, n1.w - rmax, n2.x - rmax, n2.y + rmax, n2.z + rmax, n2.w + rmax,
                          r, tmax, tn1) && r1 != r0;
        for (int c = 0; c < 2; ++c) {
            int32_t rr = c ? r1 : r0;
            bool hh = c ? h1 : h0;
            if (hh && rr < 0) {
                int32_t rx_id = __ldg(a.rx_order + (~rr));
                float4 ph = __ldg(a.rx_df + 2 * rx_id), pl = __ldg(a.rx_df + 2 * rx_id + 1);
                df3 R{df_make(ph.x, pl.x), df_make(ph.y, pl.y), df_make(ph.z, pl.z)};
                float dist;
                if (rx_accept(o, d, L, t_hit, hit, R, a2o3, dist)) {
                    uint32_t key[kKeyWords];
                    key[0] = (uint32_t)rx_id;
                    key[1] = (uint32_t)bounce;
                    for (int k = 0; k < kKmax; ++k)
                        key[2 + k] = k < bounce ? (uint32_t)a.seq[(int64_t)k * a.Rr + (ray - a.ray0)] : 0xffffffffu;
                    unsigned long long val = ((unsigned long long)__float_as_uint(dist) << 32) | ray;
                    ht_insert(a, key, val);
                    atomicAdd(&a.cnt->candidates, 1ull);
                }
                if (c) h1 = false; else h0 = false;
            }
        }
        if (h0 && h1) {
            if (sp < kStack) stack[sp++] = r1;
            else { atomicOr(&a.cnt->status, (unsigned)ST_STACK); return; }
            node = r0;
        } else if (h0) {
            node = r0;
        } else if (h1) {
            node = r1;
        } else {
            if (sp == 0) return;
            node = stack[--sp];
        }
    }
}

// ---------------------------------------------------------------- bounce kernel
__device__ __forceinline__ df3 ld_plane_n(const float4* plane, int32_t j, df& c) {
    float4 h = __ldg(plane + 2 * j), l = __ldg(plane + 2 * j + 1);
    c = df_make(h.w, l.w);
    return df3{df_make(h.x, l.x), df_make(h.y, l.y), df_make(h.z, l.z)};
}

// Final decision of a segment's closest hit after the FP32 traversal: the exact
// FP64 rule over the uncertain faces (or a full FP64 traversal when their list
// overflowed), else the certain FP32 face with t from its double-float plane.
// For a hit, nd = n.d with the face's double-float normal (the reflection
// reuses it).
template <class A>
__device__ __forceinline__ int32_t settle_hit(const A& a, const df3& o, const df3& d, int prev, const Trav& tv,
                                              int32_t j, int* stack, df& t, df& nd) {
    if (tv.overflow || tv.nu > 0) {
        d3 o64 = mk3(df_to_double(o.x), df_to_double(o.y), df_to_double(o.z));
        d3 d64 = mk3(df_to_double(d.x), df_to_double(d.y), df_to_double(d.z));
        double t64 = INFINITY;
        if (tv.overflow) {
            j = traverse64(a, o64, d64, prev, t64, stack);
            atomicAdd(&a.cnt->fp64_segments, 1ull);
        } else {
            // exact rule over the certain best and the uncertain faces
            int32_t bj = -1, bface = 0x7fffffff;
            for (int k = -1; k < tv.nu; ++k) {
                int32_t c = k < 0 ? tv.best_j : tv.unc[k];
                if (c < 0) continue;
                double tc;
                int face = __float_as_int(__ldg(a.tris + 3 * c + 1).w);
                if (mt64(a.tris, c, o64, d64, tc) && (tc < t64 || (tc == t64 && face < bface))) {
                    t64 = tc; bj = c; bface = face;
                }
            }
            j = bj;
            atomicAdd(&a.cnt->fp64_tests, (unsigned long long)(tv.nu + (tv.best_j >= 0)));
        }
        if (j >= 0) {
            t = df_from_double(t64);
            df c;
            nd = df3_dot(ld_plane_n(a.plane, j, c), d);
        }
    } else if (j >= 0) {
        df c;
        df3 n = ld_plane_n(a.plane, j, c);
        nd = df3_dot(n, d);
        t = df_div(df_sub(c, df3_dot(n, o)), nd);
    }
    return j;
}

template <bool kCount>
__global__ void __launch_bounds__(kTraceThreads, 8)
k_trace_bounce(const __grid_constant__ TraceArgs a) {
    ::sbr::pdl_wait();
    int stack[kStack];
    unsigned visits = 0, tests = 0, rx_visits = 0, edge = 0;
    const int lane = threadIdx.x & 31;
    const unsigned long long n_in = a.bounce == 0 ? (unsigned long long)a.Rr : *a.n_in;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.work, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_in) break;
        unsigned long long i = base + lane;
        bool survive = false;
        RayRec out;
        if (i < n_in) {
            df3 o, d;
            df L;
            uint32_t ray;
            int prev;
            if (a.bounce == 0) {
                ray = pool_ray(a, i);
                o = df3{df_make(a.tx_h[0], a.tx_l[0]), df_make(a.tx_h[1], a.tx_l[1]),
                        df_make(a.tx_h[2], a.tx_l[2])};
                d = geodesic_dir_df(a.ico, a.geo, ray);
                L = df_make(0.f, 0.f);
                prev = -1;
            } else {
                const RayRec* q = a.qin + i;
                const float4* q4 = reinterpret_cast<const float4*>(q);
                float4 w0 = q4[0], w1 = q4[1], w2 = q4[2], w3 = q4[3];
                o = df3{df_make(w0.x, w0.w), df_make(w0.y, w1.x), df_make(w0.z, w1.y)};
                d = df3{df_make(w1.z, w2.y), df_make(w1.w, w2.z), df_make(w2.x, w2.w)};
                L = df_make(w3.x, w3.y);
                ray = __float_as_uint(w3.z);
                prev = __float_as_int(w3.w);
            }
            Ray32 r = make_ray32(df3_hi(o), df3_hi(d));
            int32_t j = -1;
            df t = df_make(INFINITY, 0.f), nd = df_make(0.f, 0.f);
            if (a.T > 0) {
                Trav tv;
                j = traverse32<kCount>(a, r, prev, tv, stack, &visits, &tests);
                j = settle_hit(a, o, d, prev, tv, j, stack, t, nd);
            }
            if (kCount && j >= 0) {
                d3 o64 = mk3(df_to_double(o.x), df_to_double(o.y), df_to_double(o.z));
                d3 d64 = mk3(df_to_double(d.x), df_to_double(d.y), df_to_double(d.z));
                edge += min_bary64(a.tris, j, o64, d64) <= 1e-6 ? 1u : 0u;
            }
            receive<kCount>(a, a.bounce, o, d, L, t, j >= 0, r, ray, stack, &rx_visits);
            if (j >= 0 && a.bounce < a.K) {
                df c;
                df3 n = ld_plane_n(a.plane, j, c);
                int32_t surf = __float_as_int(__ldg(a.tris + 3 * j).w);
                df3 o2 = df3_fma(o, d, t);
                df dn = nd;
                df3 d2 = df3_fma(d, n, df_make(-2.f * dn.hi, -2.f * dn.lo));
                df L2 = df_add(L, t);
                out.oh[0] = o2.x.hi; out.oh[1] = o2.y.hi; out.oh[2] = o2.z.hi;
                out.ol[0] = o2.x.lo; out.ol[1] = o2.y.lo; out.ol[2] = o2.z.lo;
                out.dh[0] = d2.x.hi; out.dh[1] = d2.y.hi; out.dh[2] = d2.z.hi;
                out.dl[0] = d2.x.lo; out.dl[1] = d2.y.lo; out.dl[2] = d2.z.lo;
                out.Lh = L2.hi;
                out.Ll = L2.lo;
                out.ray = ray;
                out.prev = surf;
                a.seq[(int64_t)a.bounce * a.Rr + (ray - a.ray0)] = surf;
                a.seqf[(int64_t)a.bounce * a.Rr + (ray - a.ray0)] = __float_as_int(__ldg(a.tris + 3 * j + 1).w);
                survive = true;
            }
        }
        if (kCount) {
            unsigned long long v = visits, w = tests, x = rx_visits, e = edge;
            for (int o = 16; o; o >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
                x += __shfl_xor_sync(0xffffffffu, x, o);
                e += __shfl_xor_sync(0xffffffffu, e, o);
            }
            if (lane == 0) {
                atomicAdd(&a.cnt->node_visits, v);
                atomicAdd(&a.cnt->tri_tests, w);
                atomicAdd(&a.cnt->rx_visits, x);
                if (e) atomicAdd(&a.cnt->near_edge_hits, e);
            }
            visits = tests = rx_visits = edge = 0;
        }
        unsigned mask = __ballot_sync(0xffffffffu, survive);
        if (mask) {
            unsigned long long ob = 0;
            if (lane == 0) ob = atomicAdd(a.n_out, (unsigned long long)__popc(mask));
            ob = __shfl_sync(0xffffffffu, ob, 0);
            if (survive) {
                unsigned long long pos = ob + __popc(mask & ((1u << lane) - 1u));
                float4* q4 = reinterpret_cast<float4*>(a.qout + pos);
                q4[0] = make_float4(out.oh[0], out.oh[1], out.oh[2], out.ol[0]);
                q4[1] = make_float4(out.ol[1], out.ol[2], out.dh[0], out.dh[1]);
                q4[2] = make_float4(out.dh[2], out.dl[0], out.dl[1], out.dl[2]);
                q4[3] = make_float4(out.Lh, out.Ll, __uint_as_float(out.ray), __int_as_float(out.prev));
            }
        }
    }
}

// ---------------------------------------------------------------- depth-first tail
// From bounce a.bounce on, each lane keeps its ray's state in registers and
// traces it through every remaining bounce; a lane whose ray has ended takes the
// next ray of the input (one warp-aggregated atomic per refill), so no lane
// idles while the pool lasts and the tail needs neither queues nor launches
// per bounce. The per-segment step is the breadth-first kernel's; survivors
// are still counted per bounce (rays entering bounce b in queue[b]).
template <bool kCount>
__global__ void __launch_bounds__(kTraceThreads, 8)
k_trace_df(const __grid_constant__ TraceArgs a) {
    ::sbr::pdl_wait();
    int stack[kStack];
    // rays entering each bounce, counted per block in shared memory and added
    // to the global counters once at the end
    __shared__ unsigned s_queue[kKmax + 2];
    if (threadIdx.x < kKmax + 2) s_queue[threadIdx.x] = 0u;
    __syncthreads();
    unsigned visits = 0, tests = 0, rx_visits = 0, edge = 0;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned long long n_in = a.bounce == 0 ? (unsigned long long)a.Rr : *a.n_in;
    df3 o{}, d{};
    df L = df_make(0.f, 0.f);
    uint32_t ray = 0;
    int prev = -1, bounce = 0;
    bool has = false, exhausted = false;
    for (;;) {
        const unsigned need = __ballot_sync(FULL, !has);
        if (need && !exhausted) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.work, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (base + __popc(need) >= n_in) exhausted = true;
            if (!has) {
                const unsigned long long i = base + __popc(need & ((1u << lane) - 1u));
                if (i < n_in) {
                    if (a.bounce == 0) {
                        // launch (Sec. II-A.1): the geodesic direction decoded from the id
                        ray = pool_ray(a, i);
                        o = df3{df_make(a.tx_h[0], a.tx_l[0]), df_make(a.tx_h[1], a.tx_l[1]),
                                df_make(a.tx_h[2], a.tx_l[2])};
                        d = geodesic_dir_df(a.ico, a.geo, ray);
                        L = df_make(0.f, 0.f);
                        prev = -1;
                    } else {
                        const float4* q4 = reinterpret_cast<const float4*>(a.qin + i);
                        float4 w0 = q4[0], w1 = q4[1], w2 = q4[2], w3 = q4[3];
                        o = df3{df_make(w0.x, w0.w), df_make(w0.y, w1.x), df_make(w0.z, w1.y)};
                        d = df3{df_make(w1.z, w2.y), df_make(w1.w, w2.z), df_make(w2.x, w2.w)};
                        L = df_make(w3.x, w3.y);
                        ray = __float_as_uint(w3.z);
                        prev = __float_as_int(w3.w);
                    }
                    bounce = a.bounce;
                    has = true;
                }
            }
        }
        if (!__any_sync(FULL, has)) break;
        int entered = -1;   // bounce this lane's ray enters after this segment
        if (has) {
            Ray32 r = make_ray32(df3_hi(o), df3_hi(d));
            int32_t j = -1;
            df t = df_make(INFINITY, 0.f), nd = df_make(0.f, 0.f);
            if (a.T > 0) {
                Trav tv;
                j = traverse32<kCount>(a, r, prev, tv, stack, &visits, &tests);
                j = settle_hit(a, o, d, prev, tv, j, stack, t, nd);
            }
            if (kCount && j >= 0) {
                d3 o64 = mk3(df_to_double(o.x), df_to_double(o.y), df_to_double(o.z));
                d3 d64 = mk3(df_to_double(d.x), df_to_double(d.y), df_to_double(d.z));
                edge += min_bary64(a.tris, j, o64, d64) <= 1e-6 ? 1u : 0u;
            }
            receive<kCount>(a, bounce, o, d, L, t, j >= 0, r, ray, stack, &rx_visits);
            if (j >= 0 && bounce < a.K) {
                df c;
                df3 n = ld_plane_n(a.plane, j, c);
                int32_t surf = __float_as_int(__ldg(a.tris + 3 * j).w);
                df3 o2 = df3_fma(o, d, t);
                df dn = nd;
                d = df3_fma(d, n, df_make(-2.f * dn.hi, -2.f * dn.lo));
                o = o2;
                L = df_add(L, t);
                // per-bounce records, written once and read after the launch: streaming stores
                __stcs(&a.seq[(int64_t)bounce * a.Rr + (ray - a.ray0)], surf);
                __stcs(&a.seqf[(int64_t)bounce * a.Rr + (ray - a.ray0)], __float_as_int(__ldg(a.tris + 3 * j + 1).w));
                prev = surf;
                bounce += 1;
                entered = bounce;
            } else {
                has = false;
            }
        }
        // rays entering bounce b are counted in queue[b]: one shared atomic per
        // distinct b in the warp
        const unsigned grp = __match_any_sync(FULL, entered);
        if (entered >= 0 && lane == __ffs(grp) - 1) atomicAdd(&s_queue[entered], (unsigned)__popc(grp));
    }
    // every warp of the block leaves the loop above (no early return)
    __syncthreads();
    if (threadIdx.x < kKmax + 2 && s_queue[threadIdx.x])
        atomicAdd(&a.cnt->queue[threadIdx.x], (unsigned long long)s_queue[threadIdx.x]);
    if (kCount) {
        unsigned long long v = visits, w = tests, x = rx_visits, e = edge;
        for (int s = 16; s; s >>= 1) {
            v += __shfl_xor_sync(FULL, v, s);
            w += __shfl_xor_sync(FULL, w, s);
            x += __shfl_xor_sync(FULL, x, s);
            e += __shfl_xor_sync(FULL, e, s);
        }
        if (lane == 0) {
            atomicAdd(&a.cnt->node_visits, v);
            atomicAdd(&a.cnt->tri_tests, w);
            atomicAdd(&a.cnt->rx_visits, x);
            if (e) atomicAdd(&a.cnt->near_edge_hits, e);
        }
    }
}

// ---------------------------------------------------------------- batched bounce kernel
// The same segment step for a wave of jobs (Tx-Rx pairs over several scenes)
// in one launch per bounce: a ray's job comes from a binary search over the
// jobs' first rays at bounce 0 and from its queue record afterwards (12 bits
// split over the record's ray id and last-surface words). Each job has one
// receiver, tested exactly with the same double-float rule; the dedup key
// carries the job's index in the wave in place of the receiver index.
struct JobScene {
    const float4* nodes;
    const float4* tris;
    const float4* plane;
    TraceCountersDev* cnt;
    int64_t rot_stride;
};

struct BatchTraceArgs {
    IcoLattice ico;
    const BatchJobDev* jobs;
    const int64_t* ray_off;
    int32_t n_jobs;
    int bounce;
    int64_t R_total;
    const RayRec* qin;
    RayRec* qout;
    const unsigned long long* n_in;
    unsigned long long* n_out;
    unsigned long long* work;
    uint32_t* ht_state;
    uint32_t* ht_key;
    unsigned long long* ht_val;
    uint32_t ht_mask;
    TraceCountersDev* cnt;
};

__global__ void __launch_bounds__(kTraceThreads) k_trace_batch(const __grid_constant__ BatchTraceArgs a) {
    int stack[kStack];
    const int lane = threadIdx.x & 31;
    const unsigned long long n_in = a.bounce == 0 ? (unsigned long long)a.R_total : *a.n_in;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.work, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_in) break;
        unsigned long long i = base + lane;
        bool survive = false;
        RayRec out;
        if (i < n_in) {
            df3 o, d;
            df L;
            uint32_t ray;
            int prev, job;
            if (a.bounce == 0) {
                // the last job whose first ray is <= i
                int lo = 0, hi = a.n_jobs - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (__ldg(a.ray_off + mid) <= (int64_t)i) lo = mid; else hi = mid - 1;
                }
                job = lo;
                const BatchJobDev* J = a.jobs + job;
                ray = (uint32_t)((int64_t)i - __ldg(a.ray_off + job));
                o = df3{df_make(J->tx_h[0], J->tx_l[0]), df_make(J->tx_h[1], J->tx_l[1]),
                        df_make(J->tx_h[2], J->tx_l[2])};
                d = geodesic_dir_df(a.ico, J->geo, ray);
                L = df_make(0.f, 0.f);
                prev = -1;
            } else {
                const float4* q4 = reinterpret_cast<const float4*>(a.qin + i);
                float4 w0 = q4[0], w1 = q4[1], w2 = q4[2], w3 = q4[3];
                o = df3{df_make(w0.x, w0.w), df_make(w0.y, w1.x), df_make(w0.z, w1.y)};
                d = df3{df_make(w1.z, w2.y), df_make(w1.w, w2.z), df_make(w2.x, w2.w)};
                L = df_make(w3.x, w3.y);
                uint32_t rw = __float_as_uint(w3.z), pw = __float_as_uint(w3.w);
                ray = rw & 0xffffffu;
                prev = (int)(pw & 0x0fffffffu);
                job = (int)((rw >> 24) | ((pw >> 28) << 8));
            }
            const BatchJobDev* J = a.jobs + job;
            const JobScene sc{J->nodes, J->tris, J->plane, a.cnt, J->rot_stride};
            Ray32 r = make_ray32(df3_hi(o), df3_hi(d));
            df t = df_make(INFINITY, 0.f), nd = df_make(0.f, 0.f);
            Trav tv;
            int32_t j = traverse32<false>(sc, r, prev, tv, stack, nullptr, nullptr);
            j = settle_hit(sc, o, d, prev, tv, j, stack, t, nd);
            {
                const float4 rh = J->rx_h, rl = J->rx_l, al = J->alpha;
                const df3 Rx{df_make(rh.x, rl.x), df_make(rh.y, rl.y), df_make(rh.z, rl.z)};
                float dist;
                if (rx_accept(o, d, L, t, j >= 0, Rx, df_make(al.z, al.w), dist)) {
                    uint32_t key[kKeyWords];
                    key[0] = (uint32_t)job;
                    key[1] = (uint32_t)a.bounce;
                    for (int k = 0; k < kKmax; ++k)
                        key[2 + k] = k < a.bounce ? (uint32_t)J->seq[(int64_t)k * J->R + ray] : 0xffffffffu;
                    unsigned long long val = ((unsigned long long)__float_as_uint(dist) << 32) | ray;
                    ht_insert(a, key, val);
                    atomicAdd(&a.cnt->candidates, 1ull);
                }
            }
            if (j >= 0 && a.bounce < J->K) {
                df c;
                df3 n = ld_plane_n(J->plane, j, c);
                int32_t surf = __float_as_int(__ldg(J->tris + 3 * j).w);
                df3 o2 = df3_fma(o, d, t);
                df dn = nd;
                df3 d2 = df3_fma(d, n, df_make(-2.f * dn.hi, -2.f * dn.lo));
                df L2 = df_add(L, t);
                out.oh[0] = o2.x.hi; out.oh[1] = o2.y.hi; out.oh[2] = o2.z.hi;
                out.ol[0] = o2.x.lo; out.ol[1] = o2.y.lo; out.ol[2] = o2.z.lo;
                out.dh[0] = d2.x.hi; out.dh[1] = d2.y.hi; out.dh[2] = d2.z.hi;
                out.dl[0] = d2.x.lo; out.dl[1] = d2.y.lo; out.dl[2] = d2.z.lo;
                out.Lh = L2.hi;
                out.Ll = L2.lo;
                out.ray = ray | ((uint32_t)job << 24);
                out.prev = (int32_t)((uint32_t)surf | ((uint32_t)(job >> 8) << 28));
                J->seq[(int64_t)a.bounce * J->R + ray] = surf;
                survive = true;
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, survive);
        if (mask) {
            unsigned long long ob = 0;
            if (lane == 0) ob = atomicAdd(a.n_out, (unsigned long long)__popc(mask));
            ob = __shfl_sync(0xffffffffu, ob, 0);
            if (survive) {
                unsigned long long pos = ob + __popc(mask & ((1u << lane) - 1u));
                float4* q4 = reinterpret_cast<float4*>(a.qout + pos);
                q4[0] = make_float4(out.oh[0], out.oh[1], out.oh[2], out.ol[0]);
                q4[1] = make_float4(out.ol[1], out.ol[2], out.dh[0], out.dh[1]);
                q4[2] = make_float4(out.dh[2], out.dl[0], out.dl[1], out.dl[2]);
                q4[3] = make_float4(out.Lh, out.Ll, __uint_as_float(out.ray), __int_as_float(out.prev));
            }
        }
    }
}

// the batched step, depth first: each lane carries its ray (and job) through
// every bounce of its job, then takes the next ray of the wave
// eight 128-thread blocks per SM (64 registers), as the single-job depth-first
// kernel: the walks are latency-bound and gain more from resident warps than
// they lose to spills (4096-job batch: 2.07 s at 96 registers and 4 blocks,
// 1.64 s here)
__global__ void __launch_bounds__(kTraceThreads, 8) k_trace_batch_df(const __grid_constant__ BatchTraceArgs a) {
    int stack[kStack];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned long long n_in = (unsigned long long)a.R_total;
    df3 o{}, d{};
    df L = df_make(0.f, 0.f);
    uint32_t ray = 0;
    int prev = -1, bounce = 0, job = 0;
    bool has = false, exhausted = false;
    for (;;) {
        const unsigned need = __ballot_sync(FULL, !has);
        if (need && !exhausted) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.work, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (base + __popc(need) >= n_in) exhausted = true;
            if (!has) {
                const unsigned long long i = base + __popc(need & ((1u << lane) - 1u));
                if (i < n_in) {
                    int lo = 0, hi = a.n_jobs - 1;   // the last job whose first ray is <= i
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (__ldg(a.ray_off + mid) <= (int64_t)i) lo = mid; else hi = mid - 1;
                    }
                    job = lo;
                    const BatchJobDev* J = a.jobs + job;
                    ray = (uint32_t)((int64_t)i - __ldg(a.ray_off + job));
                    o = df3{df_make(J->tx_h[0], J->tx_l[0]), df_make(J->tx_h[1], J->tx_l[1]),
                            df_make(J->tx_h[2], J->tx_l[2])};
                    d = geodesic_dir_df(a.ico, J->geo, ray);
                    L = df_make(0.f, 0.f);
                    prev = -1;
                    bounce = 0;
                    has = true;
                }
            }
        }
        if (!__any_sync(FULL, has)) break;
        int entered = -1;
        if (has) {
            const BatchJobDev* J = a.jobs + job;
            const JobScene sc{J->nodes, J->tris, J->plane, a.cnt, J->rot_stride};
            Ray32 r = make_ray32(df3_hi(o), df3_hi(d));
            df t = df_make(INFINITY, 0.f), nd = df_make(0.f, 0.f);
            Trav tv;
            int32_t j = traverse32<false>(sc, r, prev, tv, stack, nullptr, nullptr);
            j = settle_hit(sc, o, d, prev, tv, j, stack, t, nd);
            {
                const float4 rh = J->rx_h, rl = J->rx_l, al = J->alpha;
                const df3 Rx{df_make(rh.x, rl.x), df_make(rh.y, rl.y), df_make(rh.z, rl.z)};
                float dist;
                if (rx_accept(o, d, L, t, j >= 0, Rx, df_make(al.z, al.w), dist)) {
                    uint32_t key[kKeyWords];
                    key[0] = (uint32_t)job;
                    key[1] = (uint32_t)bounce;
                    for (int k = 0; k < kKmax; ++k)
                        key[2 + k] = k < bounce ? (uint32_t)J->seq[(int64_t)k * J->R + ray] : 0xffffffffu;
                    unsigned long long val = ((unsigned long long)__float_as_uint(dist) << 32) | ray;
                    ht_insert(a, key, val);
                    atomicAdd(&a.cnt->candidates, 1ull);
                }
            }
            if (j >= 0 && bounce < J->K) {
                df c;
                df3 n = ld_plane_n(J->plane, j, c);
                int32_t surf = __float_as_int(__ldg(J->tris + 3 * j).w);
                df3 o2 = df3_fma(o, d, t);
                df dn = nd;
                d = df3_fma(d, n, df_make(-2.f * dn.hi, -2.f * dn.lo));
                o = o2;
                L = df_add(L, t);
                J->seq[(int64_t)bounce * J->R + ray] = surf;
                prev = surf;
                bounce += 1;
                entered = bounce;
            } else {
                has = false;
            }
        }
        const unsigned grp = __match_any_sync(FULL, entered);
        if (entered >= 0 && lane == __ffs(grp) - 1)
            atomicAdd(&a.cnt->queue[entered], (unsigned long long)__popc(grp));
    }
}

// Set-up of one trace in one launch: zeroed counters with queue[0] = R, an
// empty dedup table, per receiver its point box (FP32, rounded outward) and its
// double-float position, and the reception constants alpha and alpha^2 / 3 as
// double-float (alpha_in > 0 is stored to *alpha first; otherwise *alpha was
// computed on the device before this launch).
static_assert(offsetof(TraceCountersDev, queue) == 0 && sizeof(TraceCountersDev) % 8 == 0,
              "counters are 64-bit words, queue[0] first");

__global__ void k_trace_setup(TraceCountersDev* __restrict__ cnt, unsigned long long R,
                              uint32_t* __restrict__ ht_state, unsigned long long* __restrict__ ht_val,
                              size_t cap, const double* __restrict__ rx, int32_t n_rx,
                              float* __restrict__ rx_box, float4* __restrict__ rx_df, double* alpha,
                              double alpha_in, float4* __restrict__ alpha_df) {
    ::sbr::pdl_wait();
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < sizeof(TraceCountersDev) / 8) reinterpret_cast<unsigned long long*>(cnt)[i] = i == 0 ? R : 0ull;
    if (i < cap) {
        ht_state[i] = 0u;
        ht_val[i] = ~0ull;
    }
    if (i < (size_t)n_rx) {
        for (int k = 0; k < 3; ++k) {
            rx_box[6 * i + k] = __double2float_rd(rx[3 * i + k]);
            rx_box[6 * i + 3 + k] = __double2float_ru(rx[3 * i + k]);
        }
        df x = df_from_double(rx[3 * i]), y = df_from_double(rx[3 * i + 1]), z = df_from_double(rx[3 * i + 2]);
        rx_df[2 * i] = make_float4(x.hi, y.hi, z.hi, 0.f);
        rx_df[2 * i + 1] = make_float4(x.lo, y.lo, z.lo, 0.f);
    }
    if (i == 0) {
        double al = alpha_in;
        if (al > 0.0) *alpha = al;
        else al = *alpha;
        df a1 = df_from_double(al), a2 = df_from_double(al * al / 3.0);
        *alpha_df = make_float4(a1.hi, a1.lo, a2.hi, a2.lo);
    }
}

__global__ void k_init_table(uint32_t* state, unsigned long long* val, size_t cap) {
    ::sbr::pdl_wait();
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    state[i] = 0u;
    val[i] = ~0ull;
}

// ---------------------------------------------------------------- records of a trace
// The deduplicated receptions as plain records (keys, packed (dist, ray)), and
// a table rebuilt from records of several traces with the same insertion rule.
__global__ void k_entries(const uint32_t* __restrict__ state, const uint32_t* __restrict__ key,
                          const unsigned long long* __restrict__ val, size_t cap_t, uint32_t* __restrict__ out_k,
                          unsigned long long* __restrict__ out_v, int64_t cap, unsigned long long* count) {
    ::sbr::pdl_wait();
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool full = s < cap_t && state[s] == 2u;
    const unsigned m = __ballot_sync(0xffffffffu, full);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!full) return;
    const int64_t pos = (int64_t)(base + __popc(m & ((1u << lane) - 1u)));
    if (pos >= cap) return;
    for (int k = 0; k < kKeyWords; ++k) out_k[pos * kKeyWords + k] = key[s * kKeyWords + k];
    out_v[pos] = val[s];
}

struct MergeArgs {
    uint32_t* ht_state;
    uint32_t* ht_key;
    unsigned long long* ht_val;
    uint32_t ht_mask;
    TraceCountersDev* cnt;
};

__global__ void k_merge(const __grid_constant__ MergeArgs a, const uint32_t* __restrict__ keys,
                        const unsigned long long* __restrict__ vals, int64_t n) {
    ::sbr::pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t key[kKeyWords];
        for (int k = 0; k < kKeyWords; ++k) key[k] = keys[i * kKeyWords + k];
        ht_insert(a, key, vals[i]);
    }
}

// Launch order of the face rays: by the height (z) of the face's centroid on
// the icosahedron, lowest first. Rays toward the ground and the facades take
// several reflections and rays toward the sky end after one segment; with the
// sky last, the rays still in flight when the pool runs out are short, and
// fewer SMs idle while the last warps drain.
void set_pool_order(int N, TraceArgs* a) {
    const Ico ico = make_ico();
    a->pool_pre = 12 + 30 * (int64_t)(N - 1);
    a->pool_face = (int64_t)(N - 1) * (N - 2) / 2;
    int order[20];
    double cz[20];
    for (int f = 0; f < 20; ++f) {
        order[f] = f;
        cz[f] = ico.v[ico.f[f][0]][2] + ico.v[ico.f[f][1]][2] + ico.v[ico.f[f][2]][2];
    }
    std::stable_sort(order, order + 20, [&](int x, int y) { return cz[x] < cz[y]; });
    for (int f = 0; f < 20; ++f) a->face_order[f] = (uint8_t)order[f];
}

int trace_grid(bool count) {
    static int grid[2] = {0, 0};
    if (!grid[count]) {
        int per_sm = 0;
        if (count)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_bounce<true>, kTraceThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_bounce<false>, kTraceThreads, 0);
        grid[count] = std::max(1, per_sm) * sm_count();
    }
    return grid[count];
}

}  // namespace

int batch_trace_kernels(int Kmax) { return Kmax + 3; }

int batch_trace_occupancy(bool depth_first) {
    int per_sm = 0;
    cudaError_t e = depth_first
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_batch_df, kTraceThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_batch, kTraceThreads, 0);
    return e == cudaSuccess ? std::max(1, per_sm) : 1;
}

sbr_status batch_trace_wave(const BatchTraceWave& w, int blocks_per_sm, cudaStream_t s) {
    const size_t cap = (size_t)w.ht_mask + 1;
    SBR_TRY_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(TraceCountersDev), s));
    ::sbr::note_launch(), k_init_table<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(w.ht_state, w.ht_val, cap);
    SBR_TRY_CUDA(cudaGetLastError());
    SBR_TRY(set_u64(&w.cnt->queue[0], (unsigned long long)w.R_total, s));
    int per_sm = blocks_per_sm;
    if (per_sm <= 0) {
        SBR_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_batch, kTraceThreads, 0));
        per_sm = std::max(1, per_sm);
    }
    const int grid = per_sm * sm_count();
    BatchTraceArgs a{};
    a.ico = w.ico;
    a.jobs = w.jobs;
    a.ray_off = w.ray_off;
    a.n_jobs = w.n_jobs;
    a.R_total = w.R_total;
    a.ht_state = w.ht_state;
    a.ht_key = w.ht_key;
    a.ht_val = w.ht_val;
    a.ht_mask = w.ht_mask;
    a.cnt = w.cnt;
    if (w.depth_first) {
        a.bounce = 0;
        a.work = &w.cnt->work[0];
        ::sbr::note_launch(), k_trace_batch_df<<<grid, kTraceThreads, 0, s>>>(a);
        SBR_TRY_CUDA(cudaGetLastError());
        return SBR_OK;
    }
    RayRec* q0 = static_cast<RayRec*>(w.q0);
    RayRec* q1 = static_cast<RayRec*>(w.q1);
    for (int bnc = 0; bnc <= w.Kmax; ++bnc) {
        a.bounce = bnc;
        a.qin = (bnc & 1) ? q0 : q1;
        a.qout = (bnc & 1) ? q1 : q0;
        a.n_in = &w.cnt->queue[bnc];
        a.n_out = &w.cnt->queue[bnc + 1];
        a.work = &w.cnt->work[bnc];
        ::sbr::note_launch(), k_trace_batch<<<grid, kTraceThreads, 0, s>>>(a);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    return SBR_OK;
}

sbr_status trace_run(const sbr_bvh* b, sbr_trace_result* tr, cudaStream_t s) {
    const sbr_trace_params& p = tr->params;
    const int K = p.max_bounces;
    const int64_t R = tr->Rr;   // rays traced: the id range [ray0, ray0 + Rr)
    size_t cap = (size_t)1 << tr->table_log2;
    SBR_TRY(dalloc_n(&tr->ht_state, cap, s));
    SBR_TRY(dalloc_n(&tr->ht_key, cap * kKeyWords, s));
    SBR_TRY(dalloc_n(&tr->ht_val, cap, s));
    SBR_TRY(dalloc_n(&tr->cnt, 1, s));
    BvhNodes rxb;
    float* rxbox = nullptr;
    int32_t* rx_depth = nullptr;
    float4* rx_df = nullptr;
    float4* alpha_df = nullptr;
    SBR_TRY(dalloc_n(&alpha_df, 1, s));
    if (tr->n_rx > 0) {
        SBR_TRY(dalloc_n(&rxbox, 6 * (size_t)tr->n_rx, s));
        SBR_TRY(dalloc_n(&rx_depth, 1, s));
        SBR_TRY(dalloc_n(&rx_df, 2 * (size_t)tr->n_rx, s));
    }
    {
        const size_t n_set = std::max<size_t>(std::max<size_t>(cap, (size_t)tr->n_rx), sizeof(TraceCountersDev) / 8);
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_trace_setup, dim3((unsigned)((n_set + 255) / 256)), dim3(256), 0, s,
            tr->cnt, (unsigned long long)R, tr->ht_state, tr->ht_val, cap, tr->rx, tr->n_rx, rxbox, rx_df,
            tr->d_alpha, p.alpha, alpha_df);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    // receiver BVH
    if (tr->n_rx > 0) SBR_TRY(build_lbvh(rxbox, tr->n_rx, 0.0f, 1, &rxb, rx_depth, s));
    RayRec *q0 = nullptr, *q1 = nullptr;
    int32_t* seq = nullptr;
    if (K > 0) {
        if (tr->df_from > 0) {   // ray queues of the breadth-first bounces
            SBR_TRY(dalloc_n(&q0, (size_t)R, s));
            SBR_TRY(dalloc_n(&q1, (size_t)R, s));
        }
        SBR_TRY(dalloc_n(&seq, (size_t)R * K, s));
        SBR_TRY(dalloc_n(&tr->seqf, (size_t)R * K, s));
    }
    TraceArgs a{};
    a.nodes = b->tree.nodes;
    a.tris = b->tri_sorted;
    a.plane = b->plane_sorted;
    a.T = b->T;
    a.rot_stride = 3 * b->T;
    a.rx_nodes = rxb.nodes;
    a.rx_order = rxb.order;
    a.rx_df = rx_df;
    a.rx_root = rxb.d_root;
    a.n_rx = tr->n_rx;
    a.alpha_df = alpha_df;
    a.ico = make_ico_lattice();
    a.geo = make_geo_n(p.subdiv_N);
    a.N = p.subdiv_N;
    a.K = K;
    a.R = tr->R;
    a.ray0 = tr->ray0;
    a.Rr = R;
    // the whole grid is launched face by face (sky-facing faces last); a range
    // trace launches its ids in order
    if (tr->ray0 == 0 && R == tr->R) set_pool_order(p.subdiv_N, &a);
    else a.pool_pre = R, a.pool_face = 0;
    for (int k = 0; k < 3; ++k) {
        df x = df_from_double(p.tx[k]);
        a.tx_h[k] = x.hi;
        a.tx_l[k] = x.lo;
    }
    a.seq = seq;
    a.seqf = tr->seqf;
    a.ht_state = tr->ht_state;
    a.ht_key = tr->ht_key;
    a.ht_val = tr->ht_val;
    a.ht_mask = (uint32_t)(cap - 1);
    a.cnt = tr->cnt;
    const bool count = (p.flags & SBR_TRACE_COUNT_VISITS) != 0;
    int grid = trace_grid(count);
    const bool timing = (p.flags & SBR_TRACE_TIMING) != 0;
    if (timing) {
        for (int k = 0; k <= K + 1; ++k) SBR_TRY_CUDA(cudaEventCreate(&tr->ev[k]));
        SBR_TRY_CUDA(cudaEventRecord(tr->ev[0], s));
    }
    // breadth-first bounces (one launch each over a compacted queue) up to
    // df_from, then one depth-first launch for the rest
    const int df_from = std::min(K + 1, tr->df_from);
    for (int bnc = 0; bnc <= K; ++bnc) {
        a.bounce = bnc;
        a.qin = (bnc & 1) ? q0 : q1;
        a.qout = (bnc & 1) ? q1 : q0;
        a.n_in = &tr->cnt->queue[bnc];
        a.n_out = &tr->cnt->queue[bnc + 1];
        a.work = &tr->cnt->work[bnc];
        if (bnc >= df_from) {
            if (count)
                ::sbr::note_launch(), (void)::sbr::launch_pdl(k_trace_df<true>, dim3(grid), dim3(kTraceThreads), 0, s, a);
            else
                ::sbr::note_launch(), (void)::sbr::launch_pdl(k_trace_df<false>, dim3(grid), dim3(kTraceThreads), 0, s, a);
            SBR_TRY_CUDA(cudaGetLastError());
            if (timing)
                for (int k = bnc; k <= K; ++k) SBR_TRY_CUDA(cudaEventRecord(tr->ev[k + 1], s));
            break;
        }
        if (count)
            ::sbr::note_launch(), (void)::sbr::launch_pdl(k_trace_bounce<true>, dim3(grid), dim3(kTraceThreads), 0, s, a);
        else
            ::sbr::note_launch(), (void)::sbr::launch_pdl(k_trace_bounce<false>, dim3(grid), dim3(kTraceThreads), 0, s, a);
        SBR_TRY_CUDA(cudaGetLastError());
        if (timing) SBR_TRY_CUDA(cudaEventRecord(tr->ev[bnc + 1], s));
    }
    if (q0) dfree(q0, s);
    if (q1) dfree(q1, s);
    if (seq) dfree(seq, s);
    if (tr->n_rx > 0) {
        free_lbvh(&rxb, s);
        dfree(rxbox, s);
        dfree(rx_depth, s);
        dfree(rx_df, s);
    }
    dfree(alpha_df, s);
    return SBR_OK;
}

}  // namespace sbr

namespace sbr {

sbr_status trace_entries_run(const sbr_trace_result* tr, uint32_t* keys, unsigned long long* vals, int64_t cap,
                             int64_t* n_out, cudaStream_t s) {
    const size_t cap_t = (size_t)1 << tr->table_log2;
    unsigned long long* count = nullptr;
    SBR_TRY(dalloc_n(&count, 1, s));
    SBR_TRY_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_entries, dim3((unsigned)((cap_t + 255) / 256)), dim3(256), 0, s,
        tr->ht_state, tr->ht_key, tr->ht_val, cap_t, keys, vals, cap, count);
    SBR_TRY_CUDA(cudaGetLastError());
    unsigned long long h_count = 0;
    unsigned h_status = 0;
    SBR_TRY_CUDA(cudaMemcpyAsync(&h_count, count, sizeof h_count, cudaMemcpyDeviceToHost, s));
    SBR_TRY_CUDA(cudaMemcpyAsync(&h_status, &tr->cnt->status, sizeof h_status, cudaMemcpyDeviceToHost, s));
    SBR_TRY_CUDA(cudaStreamSynchronize(s));
    dfree(count, s);
    SBR_TRY(status_from_bits(h_status));
    *n_out = (int64_t)h_count;
    if ((int64_t)h_count > cap) {
        set_error("sbr_trace_entries: %lld records, buffers hold %lld", (long long)h_count, (long long)cap);
        return SBR_ERR_CAPACITY;
    }
    return SBR_OK;
}

sbr_status trace_merge_run(sbr_trace_result* tr, const uint32_t* keys, const unsigned long long* vals, int64_t n,
                           cudaStream_t s) {
    const size_t cap = (size_t)1 << tr->table_log2;
    SBR_TRY(dalloc_n(&tr->ht_state, cap, s));
    SBR_TRY(dalloc_n(&tr->ht_key, cap * kKeyWords, s));
    SBR_TRY(dalloc_n(&tr->ht_val, cap, s));
    SBR_TRY(dalloc_n(&tr->cnt, 1, s));
    SBR_TRY_CUDA(cudaMemsetAsync(tr->cnt, 0, sizeof(TraceCountersDev), s));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_init_table, dim3((unsigned)((cap + 255) / 256)), dim3(256), 0, s, tr->ht_state, tr->ht_val, cap);
    SBR_TRY_CUDA(cudaGetLastError());
    if (tr->params.alpha > 0.0) {
        unsigned long long bits;
        const double al = tr->params.alpha;
        memcpy(&bits, &al, sizeof bits);
        SBR_TRY(set_u64(reinterpret_cast<unsigned long long*>(tr->d_alpha), bits, s));
    }
    if (n > 0) {
        MergeArgs a{tr->ht_state, tr->ht_key, tr->ht_val, (uint32_t)(cap - 1), tr->cnt};
        const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 8 * (int64_t)sm_count());
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_merge, dim3(grid), dim3(256), 0, s, a, keys, vals, n);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    return SBR_OK;
}

}  // namespace sbr
