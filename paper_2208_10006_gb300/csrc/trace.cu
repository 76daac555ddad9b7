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
// The ray state (origin, direction, L) is kept in FP64 so that the hit and
// reception decisions agree with an FP64 evaluation of the same rule to
// rounding; the FP32 traversal carries the per-triangle cost.
#include <algorithm>
#include <cmath>

#include "geodesic.cuh"

namespace sbr {
namespace {

constexpr int kStack = 64;
constexpr float kCert = 1e-3f;         // relative margin below which FP32 is not trusted
constexpr int kTraceThreads = 128;
constexpr int kSpinLimit = 1 << 20;    // bounded wait for a dedup slot being published

struct RayRec {
    double o[3];
    double d[3];
    double L;
    uint32_t ray;
    int32_t prev;
};
static_assert(sizeof(RayRec) == 64, "ray record is one 64-byte line");

struct TraceArgs {
    const float4* nodes;
    const float4* tris;
    const double* nrm;
    int64_t T;
    const float4* rx_nodes;
    const int32_t* rx_order;
    const double* rx;
    const float* rx_root;
    int32_t n_rx;
    const double* alpha;
    int N, K, bounce;
    int64_t R;
    double tx[3];
    const RayRec* qin;
    RayRec* qout;
    const unsigned long long* n_in;
    unsigned long long* n_out;
    unsigned long long* work;
    int32_t* seq;
    uint32_t* ht_state;
    uint32_t* ht_key;
    unsigned long long* ht_val;
    uint32_t ht_mask;
    TraceCountersDev* cnt;
};

__device__ __forceinline__ float comp(float4 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
__device__ __forceinline__ float comp3(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

struct Ray32 {
    float3 o, d, inv;
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

__device__ __forceinline__ Ray32 make_ray32(d3 o, d3 d) {
    Ray32 r;
    r.o = make_float3((float)o.x, (float)o.y, (float)o.z);
    r.d = make_float3((float)d.x, (float)d.y, (float)d.z);
    r.inv = make_float3(1.0f / r.d.x, 1.0f / r.d.y, 1.0f / r.d.z);
    float ax = fabsf(r.d.x), ay = fabsf(r.d.y), az = fabsf(r.d.z);
    r.kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    r.kx = r.kz == 2 ? 0 : r.kz + 1;
    r.ky = r.kx == 2 ? 0 : r.kx + 1;
    float dz = comp3(r.d, r.kz);
    if (dz < 0.f) { int t = r.kx; r.kx = r.ky; r.ky = t; }
    r.Sx = comp3(r.d, r.kx) / dz;
    r.Sy = comp3(r.d, r.ky) / dz;
    r.Sz = 1.0f / dz;
    return r;
}

// slab test; NaN from 0 * inf is ignored by fminf/fmaxf, which keeps it conservative
__device__ __forceinline__ bool box_hit(float lx, float ly, float lz, float hx, float hy, float hz,
                                        const Ray32& r, float tmax, float& tnear) {
    float t0x = (lx - r.o.x) * r.inv.x, t1x = (hx - r.o.x) * r.inv.x;
    float t0y = (ly - r.o.y) * r.inv.y, t1y = (hy - r.o.y) * r.inv.y;
    float t0z = (lz - r.o.z) * r.inv.z, t1z = (hz - r.o.z) * r.inv.z;
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
// the rounding of the FP64 ray to FP32. A face is a certain miss if some edge
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
    float Ax = comp(a, r.kx) - comp3(r.o, r.kx), Ay = comp(a, r.ky) - comp3(r.o, r.ky),
          Az = comp(a, r.kz) - comp3(r.o, r.kz);
    float Bx = comp(b, r.kx) - comp3(r.o, r.kx), By = comp(b, r.ky) - comp3(r.o, r.ky),
          Bz = comp(b, r.kz) - comp3(r.o, r.kz);
    float Cx = comp(c, r.kx) - comp3(r.o, r.kx), Cy = comp(c, r.ky) - comp3(r.o, r.ky),
          Cz = comp(c, r.kz) - comp3(r.o, r.kz);
    Ax = fmaf(-r.Sx, Az, Ax); Ay = fmaf(-r.Sy, Az, Ay);
    Bx = fmaf(-r.Sx, Bz, Bx); By = fmaf(-r.Sy, Bz, By);
    Cx = fmaf(-r.Sx, Cz, Cx); Cy = fmaf(-r.Sy, Cz, Cy);
    float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
    float det = U + V + W;
    float sg = det >= 0.f ? 1.f : -1.f;
    float mn = fminf(fminf(sg * U, sg * V), sg * W);  // min of the orientation-adjusted values
    float pU = fabsf(Cx * By) + fabsf(Cy * Bx), pV = fabsf(Ax * Cy) + fabsf(Ay * Cx),
          pW = fabsf(Bx * Ay) + fabsf(By * Ax);
    float per = fabsf(Bx - Cx) + fabsf(By - Cy) + fabsf(Cx - Ax) + fabsf(Cy - Ay) +
                fabsf(Ax - Bx) + fabsf(Ay - By);
    float zs = fmaxf(fabsf(Az), fmaxf(fabsf(Bz), fabsf(Cz)));
    float errE = 8.f * kEps32 * fmaxf(pU, fmaxf(pV, pW)) + 4.f * kEps32 * (tv.omax + zs) * per;
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
// (or -1) and the list of faces that FP64 must re-decide.
__device__ int32_t traverse32(const TraceArgs& a, const Ray32& r, int prev, Trav& tv, int* stack) {
    tv.best_t = INFINITY; tv.lim = INFINITY; tv.best_j = -1; tv.best_face = 0x7fffffff;
    tv.best_surf = -2; tv.nu = 0; tv.overflow = false;
    tv.omax = fmaxf(fabsf(r.o.x), fmaxf(fabsf(r.o.y), fabsf(r.o.z)));
    int sp = 0;
    int32_t node = 0;
    for (;;) {
        const float4* nd = a.nodes + 4 * (int64_t)node;
        float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        int32_t r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
        float tn0, tn1;
        bool h0 = box_hit(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, r, tv.lim, tn0);
        bool h1 = box_hit(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, r, tv.lim, tn1) && r1 != r0;
        if (h0 && r0 < 0) { tri_test32(a.tris, ~r0, prev, r, tv); h0 = false; }
        if (h1 && r1 < 0) { tri_test32(a.tris, ~r1, prev, r, tv); h1 = false; }
        if (h0 && h1) {
            int32_t nearn = tn0 <= tn1 ? r0 : r1, farn = tn0 <= tn1 ? r1 : r0;
            if (sp < kStack) stack[sp++] = farn;
            else { atomicOr(&a.cnt->status, (unsigned)ST_STACK); tv.overflow = true; break; }
            node = nearn;
        } else if (h0) {
            node = r0;
        } else if (h1) {
            node = r1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
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

__device__ __forceinline__ bool box_hit64(const float* b, d3 o, d3 inv, double tmax) {
    double t0x = ((double)b[0] - o.x) * inv.x, t1x = ((double)b[3] - o.x) * inv.x;
    double t0y = ((double)b[1] - o.y) * inv.y, t1y = ((double)b[4] - o.y) * inv.y;
    double t0z = ((double)b[2] - o.z) * inv.z, t1z = ((double)b[5] - o.z) * inv.z;
    double tmin = fmax(fmax(fmin(t0x, t1x), fmin(t0y, t1y)), fmax(fmin(t0z, t1z), 0.0));
    double tmx = fmin(fmin(fmax(t0x, t1x), fmax(t0y, t1y)), fmin(fmax(t0z, t1z), tmax));
    return tmin <= tmx;
}

__device__ __noinline__ int32_t traverse64(const TraceArgs& a, d3 o, d3 d, int prev, double& t_out,
                                           int* stack) {
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
                int32_t j = ~rr;
                float4 a0 = __ldg(a.tris + 3 * j), a1 = __ldg(a.tris + 3 * j + 1);
                if (__float_as_int(a0.w) != prev) {
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

__device__ void ht_insert(const TraceArgs& a, const uint32_t* key, unsigned long long val) {
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
__device__ void receive(const TraceArgs& a, d3 o, d3 d, double L, double t_hit, bool hit,
                        const Ray32& r, uint32_t ray, int* stack) {
    if (a.n_rx <= 0) return;
    const double alpha = *a.alpha;
    const double inv_sqrt3 = 0.57735026918962576451;
    double t_end = t_hit;
    if (!hit) {
        // no receiver lies beyond the farthest corner of their bounding box
        double far2 = 0;
        for (int c = 0; c < 8; ++c) {
            double x = a.rx_root[(c & 1) ? 3 : 0] - o.x;
            double y = a.rx_root[(c & 2) ? 4 : 1] - o.y;
            double z = a.rx_root[(c & 4) ? 5 : 2] - o.z;
            far2 = fmax(far2, x * x + y * y + z * z);
        }
        t_end = sqrt(far2) * (1.0 + 1e-6) + 1e-3;
    }
    float rmax = (float)(alpha * (L + t_end) * inv_sqrt3 * (1.0 + 1e-5)) +
                 1e-5f * (float)(fabs(o.x) + fabs(o.y) + fabs(o.z) + L + t_end);
    float tmax = (float)(t_end * (1.0 + 1e-5)) + rmax;
    int sp = 0;
    int32_t node = 0;
    for (;;) {
        const float4* nd = a.rx_nodes + 4 * (int64_t)node;
        float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        int32_t r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
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
                d3 R = mk3(a.rx[3 * rx_id], a.rx[3 * rx_id + 1], a.rx[3 * rx_id + 2]);
                double ts = dot(R - o, d);
                if (ts >= 0.0 && ts <= t_hit) {
                    d3 p = o + d * ts;
                    double dist = norm(p - R);
                    double rad = alpha * (L + ts) * inv_sqrt3;
                    if (dist <= rad) {
                        uint32_t key[kKeyWords];
                        key[0] = (uint32_t)rx_id;
                        key[1] = (uint32_t)a.bounce;
                        for (int k = 0; k < kKmax; ++k)
                            key[2 + k] = k < a.bounce ? (uint32_t)a.seq[(int64_t)k * a.R + ray] : 0xffffffffu;
                        unsigned long long val =
                            ((unsigned long long)__float_as_uint((float)dist) << 32) | ray;
                        ht_insert(a, key, val);
                        atomicAdd(&a.cnt->candidates, 1ull);
                    }
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
__global__ void __launch_bounds__(kTraceThreads)
k_trace_bounce(const __grid_constant__ TraceArgs a, const __grid_constant__ Ico ico) {
    int stack[kStack];
    const int lane = threadIdx.x & 31;
    const unsigned long long n_in = a.bounce == 0 ? (unsigned long long)a.R : *a.n_in;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.work, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_in) break;
        unsigned long long i = base + lane;
        bool survive = false;
        RayRec out;
        if (i < n_in) {
            d3 o, d;
            double L;
            uint32_t ray;
            int prev;
            if (a.bounce == 0) {
                ray = (uint32_t)i;
                o = mk3(a.tx[0], a.tx[1], a.tx[2]);
                d = geodesic_dir(ico, a.N, ray);
                L = 0.0;
                prev = -1;
            } else {
                const RayRec* q = a.qin + i;
                o = ld3(q->o);
                d = ld3(q->d);
                L = q->L;
                ray = q->ray;
                prev = q->prev;
            }
            Ray32 r = make_ray32(o, d);
            int32_t j = -1;
            double t64 = INFINITY;
            if (a.T > 0) {
                Trav tv;
                j = traverse32(a, r, prev, tv, stack);
                if (tv.overflow) {
                    j = traverse64(a, o, d, prev, t64, stack);
                    atomicAdd(&a.cnt->fp64_segments, 1ull);
                } else if (tv.nu > 0) {
                    // exact rule over the certain best and the uncertain faces
                    int32_t bj = -1, bface = 0x7fffffff;
                    double bt = INFINITY;
                    for (int k = -1; k < tv.nu; ++k) {
                        int32_t c = k < 0 ? tv.best_j : tv.unc[k];
                        if (c < 0) continue;
                        double tc;
                        int face = __float_as_int(__ldg(a.tris + 3 * c + 1).w);
                        if (mt64(a.tris, c, o, d, tc) && (tc < bt || (tc == bt && face < bface))) {
                            bt = tc; bj = c; bface = face;
                        }
                    }
                    j = bj;
                    t64 = bt;
                    atomicAdd(&a.cnt->fp64_tests, (unsigned long long)(tv.nu + (tv.best_j >= 0)));
                } else if (j >= 0) {
                    d3 n = ld3(a.nrm + 3 * (int64_t)j);
                    float4 v0 = __ldg(a.tris + 3 * j);
                    t64 = dot(n, mk3(v0.x, v0.y, v0.z) - o) / dot(n, d);
                }
            }
            receive(a, o, d, L, t64, j >= 0, r, ray, stack);
            if (j >= 0 && a.bounce < a.K) {
                d3 n = ld3(a.nrm + 3 * (int64_t)j);
                int32_t surf = __float_as_int(__ldg(a.tris + 3 * j).w);
                d3 o2 = o + d * t64;
                d3 d2 = d - n * (2.0 * dot(d, n));
                st3(out.o, o2);
                st3(out.d, d2);
                out.L = L + t64;
                out.ray = ray;
                out.prev = surf;
                a.seq[(int64_t)a.bounce * a.R + ray] = surf;
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
                a.qout[pos] = out;
            }
        }
    }
}

__global__ void k_rx_boxes(const double* __restrict__ rx, int32_t n, float* __restrict__ box) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 3; ++k) {
        box[6 * i + k] = __double2float_rd(rx[3 * i + k]);
        box[6 * i + 3 + k] = __double2float_ru(rx[3 * i + k]);
    }
}

__global__ void k_init_table(uint32_t* state, unsigned long long* val, size_t cap) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    state[i] = 0u;
    val[i] = ~0ull;
}

int trace_grid() {
    static int grid = 0;
    if (!grid) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_bounce, kTraceThreads, 0);
        grid = std::max(1, per_sm) * sm_count();
    }
    return grid;
}

}  // namespace

sbr_status trace_run(const sbr_bvh* b, sbr_trace_result* tr, cudaStream_t s) {
    const sbr_trace_params& p = tr->params;
    const int K = p.max_bounces;
    const int64_t R = tr->R;
    size_t cap = (size_t)1 << tr->table_log2;
    SBR_TRY(dalloc_n(&tr->ht_state, cap, s));
    SBR_TRY(dalloc_n(&tr->ht_key, cap * kKeyWords, s));
    SBR_TRY(dalloc_n(&tr->ht_val, cap, s));
    SBR_TRY(dalloc_n(&tr->cnt, 1, s));
    SBR_TRY_CUDA(cudaMemsetAsync(tr->cnt, 0, sizeof(TraceCountersDev), s));
    ::sbr::note_launch(), k_init_table<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(tr->ht_state, tr->ht_val, cap);
    SBR_TRY_CUDA(cudaGetLastError());
    SBR_TRY(set_u64(&tr->cnt->queue[0], (unsigned long long)R, s));
    // receiver BVH
    BvhNodes rxb;
    float* rxbox = nullptr;
    int32_t* rx_depth = nullptr;
    if (tr->n_rx > 0) {
        SBR_TRY(dalloc_n(&rxbox, 6 * (size_t)tr->n_rx, s));
        SBR_TRY(dalloc_n(&rx_depth, 1, s));
        ::sbr::note_launch(), k_rx_boxes<<<(tr->n_rx + 255) / 256, 256, 0, s>>>(tr->rx, tr->n_rx, rxbox);
        SBR_TRY_CUDA(cudaGetLastError());
        SBR_TRY(build_lbvh(rxbox, tr->n_rx, 0.0f, &rxb, rx_depth, s));
    }
    RayRec *q0 = nullptr, *q1 = nullptr;
    int32_t* seq = nullptr;
    if (K > 0) {
        SBR_TRY(dalloc_n(&q0, (size_t)R, s));
        SBR_TRY(dalloc_n(&q1, (size_t)R, s));
        SBR_TRY(dalloc_n(&seq, (size_t)R * K, s));
    }
    TraceArgs a{};
    a.nodes = b->tree.nodes;
    a.tris = b->tri_sorted;
    a.nrm = b->nrm_sorted;
    a.T = b->T;
    a.rx_nodes = rxb.nodes;
    a.rx_order = rxb.order;
    a.rx = tr->rx;
    a.rx_root = rxb.d_root;
    a.n_rx = tr->n_rx;
    a.alpha = tr->d_alpha;
    a.N = p.subdiv_N;
    a.K = K;
    a.R = R;
    for (int k = 0; k < 3; ++k) a.tx[k] = p.tx[k];
    a.seq = seq;
    a.ht_state = tr->ht_state;
    a.ht_key = tr->ht_key;
    a.ht_val = tr->ht_val;
    a.ht_mask = (uint32_t)(cap - 1);
    a.cnt = tr->cnt;
    Ico ico = make_ico();
    int grid = trace_grid();
    const bool timing = (p.flags & SBR_TRACE_TIMING) != 0;
    if (timing) {
        for (int k = 0; k <= K + 1; ++k) SBR_TRY_CUDA(cudaEventCreate(&tr->ev[k]));
        SBR_TRY_CUDA(cudaEventRecord(tr->ev[0], s));
    }
    for (int bnc = 0; bnc <= K; ++bnc) {
        a.bounce = bnc;
        a.qin = (bnc & 1) ? q0 : q1;
        a.qout = (bnc & 1) ? q1 : q0;
        a.n_in = &tr->cnt->queue[bnc];
        a.n_out = &tr->cnt->queue[bnc + 1];
        a.work = &tr->cnt->work[bnc];
        ::sbr::note_launch(), k_trace_bounce<<<grid, kTraceThreads, 0, s>>>(a, ico);
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
    }
    return SBR_OK;
}

}  // namespace sbr
