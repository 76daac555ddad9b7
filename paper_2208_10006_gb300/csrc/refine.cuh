// Image-method refinement of one dedup key (Sec. I, image method), shared by
// the single-job and batched path kernels:
//   mirror the Tx through the surface planes in order (I_0 = Tx,
//   I_k = I_{k-1} - 2 (n_k.I_{k-1} - c_k) n_k), back-trace from the Rx
//   (P_m on segment I_m -> Rx, P_k on segment I_k -> P_{k+1}), require each
//   segment parameter in (0, 1) and each P_k inside one of its surface's
//   triangles (barycentric tolerance 1e-9), report the lowest-id such face,
//   and L = |I_m - Rx|. The plane of a surface is that of its lowest-id face.
#pragma once
#include "sbr_internal.cuh"

namespace sbr {
namespace {

__device__ __forceinline__ bool point_in_tri(const float* v, d3 p, double tol) {
    d3 a = mk3(v[0], v[1], v[2]), b = mk3(v[3], v[4], v[5]), c = mk3(v[6], v[7], v[8]);
    d3 e1 = b - a, e2 = c - a, w = p - a;
    double d00 = dot(e1, e1), d01 = dot(e1, e2), d11 = dot(e2, e2);
    double d20 = dot(w, e1), d21 = dot(w, e2);
    double den = d00 * d11 - d01 * d01;
    if (den == 0.0) return false;
    double l1 = (d11 * d20 - d01 * d21) / den;
    double l2 = (d00 * d21 - d01 * d20) / den;
    double l0 = 1.0 - l1 - l2;
    return l0 >= -tol && l1 >= -tol && l2 >= -tol;
}

// smallest FP64 barycentric of p in the face (the containment margin)
__device__ __forceinline__ double bary_margin(const float* v, d3 p) {
    d3 a = mk3(v[0], v[1], v[2]), b = mk3(v[3], v[4], v[5]), c = mk3(v[6], v[7], v[8]);
    d3 e1 = b - a, e2 = c - a, w = p - a;
    double d00 = dot(e1, e1), d01 = dot(e1, e2), d11 = dot(e2, e2);
    double d20 = dot(w, e1), d21 = dot(w, e2);
    double den = d00 * d11 - d01 * d01;
    if (den == 0.0) return -1.0;
    double l1 = (d11 * d20 - d01 * d21) / den;
    double l2 = (d00 * d21 - d01 * d20) / den;
    return fmin(fmin(l1, l2), 1.0 - l1 - l2);
}

// FP32 screen of the same barycentric test: +1 clearly inside, -1 clearly
// outside, 0 near an edge (then the FP64 test decides). The margin is 1e-3 or,
// for small or thin faces far from the origin, a bound on the FP32 error of
// the barycentrics (rounding of p and of the products, ~ eps (|a| + |w|) / (size sin^2)).
__device__ __forceinline__ int screen_in_tri(const float* v, float3 p, float extra = 0.f) {
    float3 a = make_float3(v[0], v[1], v[2]);
    float3 e1 = make_float3(v[3] - a.x, v[4] - a.y, v[5] - a.z);
    float3 e2 = make_float3(v[6] - a.x, v[7] - a.y, v[8] - a.z);
    float3 w = make_float3(p.x - a.x, p.y - a.y, p.z - a.z);
    float d00 = e1.x * e1.x + e1.y * e1.y + e1.z * e1.z, d01 = e1.x * e2.x + e1.y * e2.y + e1.z * e2.z;
    float d11 = e2.x * e2.x + e2.y * e2.y + e2.z * e2.z;
    float d20 = w.x * e1.x + w.y * e1.y + w.z * e1.z, d21 = w.x * e2.x + w.y * e2.y + w.z * e2.z;
    float den = d00 * d11 - d01 * d01;
    if (!(den > 0.f)) return 0;
    float l1 = (d11 * d20 - d01 * d21) / den, l2 = (d00 * d21 - d01 * d20) / den;
    float m = fminf(fminf(l1, l2), 1.f - l1 - l2);
    float ext = fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fabsf(a.z)) +
                fmaxf(fmaxf(fabsf(w.x), fabsf(w.y)), fabsf(w.z)) + 1.f;
    float s2 = d00 + d11;
    float margin = fmaxf(1e-3f, 16.f * 5.9604645e-8f * ext * s2 * sqrtf(s2) / den);
    return m > margin + extra ? 1 : (m < -margin ? -1 : 0);
}

// the kept ray's hit face holds the refined point by a barycentric margin of at
// least 1e-6: the FP32 screen accepts it when its margin exceeds the screen's
// error bound by 1e-6 (then the FP64 margin does too); otherwise the FP64
// margin decides
__device__ __forceinline__ bool hint_holds(const float* v, d3 p) {
    if (screen_in_tri(v, make_float3((float)p.x, (float)p.y, (float)p.z), 1e-6f) > 0) return true;
    return bary_margin(v, p) >= 1e-6;
}

__device__ __forceinline__ void angles_deg(d3 v, double* out) {
    out[0] = atan2(v.y, v.x) * (180.0 / kPi);
    out[1] = atan2(v.z, hypot(v.x, v.y)) * (180.0 / kPi);
}

// theta-hat (V) or phi-hat (H) of a unit propagation direction d, from
// cos(theta) = z, sin(theta) = rho = |(x, y)|, cos(phi) = x / rho,
// sin(phi) = y / rho; at the poles (rho = 0) phi = atan2(0, 0) = 0
__device__ __forceinline__ d3 pol_vec(d3 d, int pol) {
    double rho = hypot(d.x, d.y);
    double cp = 1.0, sp = 0.0;
    if (rho > 0.0) { cp = d.x / rho; sp = d.y / rho; }
    double ct = d.z / norm(d), st = rho / norm(d);
    if (pol == SBR_POL_V) return mk3(ct * cp, ct * sp, -st);
    return mk3(-sp, cp, 0.0);
}

// s = unit(d_in x n); when d_in is parallel to n, unit(n x e) with e the axis of
// the smallest |n| component (first on ties)
__device__ __forceinline__ d3 s_vector(d3 din, d3 n) {
    d3 cr = cross(din, n);
    double l = norm(cr);
    if (l > 1e-12) return cr * (1.0 / l);
    double ax = fabs(n.x), ay = fabs(n.y), az = fabs(n.z);
    d3 e = mk3(1, 0, 0);
    if (ay < ax && ay <= az) e = mk3(0, 1, 0);
    else if (az < ax && az < ay) e = mk3(0, 0, 1);
    return unit(cross(n, e));
}

// scene in face order: FP32 vertices, FP64 unit normals, CSR of faces per surface
struct RefineScene {
    const float* tri;
    const double* nrm;
    const int32_t* s_off;
    const int32_t* s_tri;
    int32_t S;
    const float4* nodes;   // scene BVH (null: containers are found by scanning the surface)
    const float4* tris;    // BVH-order faces: v0 (w = surface id bits), v1 (w = face id bits), v2
};

// Lowest-id face of surface s that contains p by the scan's rule (the FP32
// screen, else the FP64 test with tolerance 1e-9), from a point query of the
// scene BVH instead of a scan of the surface: a face that passes the rule holds
// p within 1e-9 of its barycentrics, far inside the padding of its BVH box, so
// the query meets every such face. -1: none; -2: the query's stack overflowed
// (the caller then scans the surface).
constexpr int kFindStack = 64;

__device__ __forceinline__ bool in_box(float3 p, float lx, float ly, float lz, float hx, float hy, float hz) {
    return p.x >= lx && p.x <= hx && p.y >= ly && p.y <= hy && p.z >= lz && p.z <= hz;
}

__device__ int32_t bvh_find_face(const RefineScene& sc, int s, d3 P) {
    const float3 pf = make_float3((float)P.x, (float)P.y, (float)P.z);
    int32_t best = 0x7fffffff;
    int32_t stack[kFindStack];
    int sp = 0;
    int32_t ref = 0;
    for (;;) {
        if (ref >= 0) {
            const float4* nd = sc.nodes + 4 * (int64_t)ref;
            const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            const int32_t r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
            const bool h0 = in_box(pf, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
            const bool h1 = in_box(pf, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w) && r1 != r0;
            if (h0 && h1) {
                if (sp == kFindStack) return -2;
                stack[sp++] = r1;
                ref = r0;
                continue;
            }
            if (h0) { ref = r0; continue; }
            if (h1) { ref = r1; continue; }
        } else {
            const int32_t first = leaf_first(ref), cnt = leaf_count(ref);
            for (int32_t j = first; j < first + cnt; ++j) {
                if (__float_as_int(__ldg(sc.tris + 3 * (int64_t)j).w) != s) continue;
                const int32_t face = __float_as_int(__ldg(sc.tris + 3 * (int64_t)j + 1).w);
                if (face >= best) continue;
                const float* v = sc.tri + 9 * (int64_t)face;
                const int scr = screen_in_tri(v, pf);
                if (scr > 0 || (scr == 0 && point_in_tri(v, P, 1e-9))) best = face;
            }
        }
        if (sp == 0) break;
        ref = stack[--sp];
    }
    return best == 0x7fffffff ? -1 : best;
}

// outputs of one refined key, written at record i (lane 0, valid keys only)
struct RefineOut {
    int32_t* nb_o;
    int32_t* surf_o;
    int32_t* face_o;
    double* pts_o;
    double* L_o;
    double* aod_o;
    double* aoa_o;
    uint32_t* ray_o;
    float* dist_o;
    double* jones_o;
};

// One key, by one warp (kSolo false: lane 0 builds the images and points,
// which the lanes share for a scan of the surface's faces 32 at a time) or by
// one thread (kSolo true: 32 keys per warp; a reflection its hint does not
// settle gets the whole warp's scan; must be called by all 32 lanes). m reflections with
// surfaces seq[0..m), kept (dist, ray) value v. hint (or null): the faces the
// kept ray hit, hint[k * hint_stride] for reflection k; a face of the surface
// that contains the point by a barycentric margin of at least 1e-6 is its only
// container (the faces of a surface do not overlap), so it is taken without
// scanning; otherwise the lowest-id container is searched. Both arrangements
// give the same result. Returns the key's validity (on every lane).
template <bool kSolo>
__device__ bool refine_key(int lane, int m, const int32_t* seq, unsigned long long v, const RefineScene& sc,
                           d3 Tx, d3 Rx, const RefineOut& o, int64_t i, const int32_t* hint = nullptr,
                           int64_t hint_stride = 0) {
    d3 nn[kKmax + 1], img[kKmax + 1], P[kKmax + 2];
    double cc[kKmax + 1];
    bool ok = m >= 0 && m <= kKmax;
    // the image construction and back-trace (FP64, scarce on this GPU) run on
    // lane 0 alone; the points are then broadcast for the containment scan
    if (kSolo || lane == 0) {
    img[0] = Tx;
    for (int k = 1; k <= m && ok; ++k) {
        int s = seq[k - 1];
        if (s < 0 || s >= sc.S || sc.s_off[s] == sc.s_off[s + 1]) { ok = false; break; }
        int32_t t0 = sc.s_tri[sc.s_off[s]];
        nn[k] = ld3(sc.nrm + 3 * (int64_t)t0);
        cc[k] = dot(nn[k], mk3(sc.tri[9 * (int64_t)t0], sc.tri[9 * (int64_t)t0 + 1], sc.tri[9 * (int64_t)t0 + 2]));
        img[k] = img[k - 1] - nn[k] * (2.0 * (dot(nn[k], img[k - 1]) - cc[k]));
    }
    d3 target = Rx;
    for (int k = m; k >= 1 && ok; --k) {
        d3 dv = target - img[k];
        double den = dot(nn[k], dv);
        if (den == 0.0) { ok = false; break; }
        double u = (cc[k] - dot(nn[k], img[k])) / den;
        if (!(u > 0.0 && u < 1.0)) { ok = false; break; }
        P[k] = img[k] + dv * u;
        target = P[k];
    }
    }
    if (!kSolo) {
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
            for (int k = 1; k <= m; ++k) {
                P[k].x = __shfl_sync(0xffffffffu, P[k].x, 0);
                P[k].y = __shfl_sync(0xffffffffu, P[k].y, 0);
                P[k].z = __shfl_sync(0xffffffffu, P[k].z, 0);
            }
        }
    }
    int32_t face[kKmax];
    for (int k = 0; k < kKmax; ++k) face[k] = -1;
    if (kSolo) {
        // every lane holds its own key; lanes whose hint does not settle a
        // reflection are served in turn by the whole warp's 32-wide scan (all
        // 32 lanes run this loop, keyless lanes with ok false)
        for (int k = 1; k <= kKmax; ++k) {
            const bool act = ok && k <= m;
            const int s = act ? seq[k - 1] : 0;
            int32_t found = -1;
            bool need = false;
            if (act) {
                const int32_t h = hint ? hint[(int64_t)(k - 1) * hint_stride] : -1;
                if (h >= 0 && hint_holds(sc.tri + 9 * (int64_t)h, P[k])) {
                    found = h;
                } else if (sc.nodes) {
                    found = bvh_find_face(sc, s, P[k]);
                    need = found == -2;
                } else {
                    need = true;
                }
            }
            unsigned nm = __ballot_sync(0xffffffffu, need);
            const double px = act ? P[k].x : 0.0, py = act ? P[k].y : 0.0, pz = act ? P[k].z : 0.0;
            while (nm) {
                const int L = __ffs(nm) - 1;
                nm &= nm - 1;
                const d3 PL = mk3(__shfl_sync(0xffffffffu, px, L), __shfl_sync(0xffffffffu, py, L),
                                  __shfl_sync(0xffffffffu, pz, L));
                const int sL = __shfl_sync(0xffffffffu, s, L);
                const float3 pf = make_float3((float)PL.x, (float)PL.y, (float)PL.z);
                const int32_t qa = sc.s_off[sL], qb = sc.s_off[sL + 1];
                int32_t fL = -1;
                for (int32_t base = qa; base < qb; base += 32) {
                    int32_t q = base + lane;
                    bool in = false;
                    if (q < qb) {
                        const float* v = sc.tri + 9 * (int64_t)sc.s_tri[q];
                        int scr = screen_in_tri(v, pf);
                        in = scr > 0 || (scr == 0 && point_in_tri(v, PL, 1e-9));
                    }
                    unsigned m32 = __ballot_sync(0xffffffffu, in);
                    if (m32) {  // faces in ascending id: the lowest lane is the lowest id
                        fL = sc.s_tri[base + __ffs(m32) - 1];
                        break;
                    }
                }
                if (lane == L) found = fL;
            }
            if (act) {
                if (found < 0) ok = false;
                else face[k - 1] = found;
            }
        }
    } else {
        for (int k = 1; k <= m && ok; ++k) {
            int s = seq[k - 1];
            int32_t found = -1;
            if (hint) {
                const int32_t h = hint[(int64_t)(k - 1) * hint_stride];
                if (h >= 0 && hint_holds(sc.tri + 9 * (int64_t)h, P[k])) {
                    face[k - 1] = h;
                    continue;
                }
            }
            if (sc.nodes) {
                int32_t f = 0;
                if (lane == 0) f = bvh_find_face(sc, s, P[k]);
                f = __shfl_sync(0xffffffffu, f, 0);
                if (f != -2) {
                    if (f < 0) { ok = false; break; }
                    face[k - 1] = f;
                    continue;
                }
            }
            const int32_t qa = sc.s_off[s], qb = sc.s_off[s + 1];
            const float3 pf = make_float3((float)P[k].x, (float)P[k].y, (float)P[k].z);
            for (int32_t base = qa; base < qb; base += 32) {
                int32_t q = base + lane;
                bool in = false;
                if (q < qb) {
                    const float* v = sc.tri + 9 * (int64_t)sc.s_tri[q];
                    int scr = screen_in_tri(v, pf);
                    in = scr > 0 || (scr == 0 && point_in_tri(v, P[k], 1e-9));
                }
                unsigned m32 = __ballot_sync(0xffffffffu, in);
                if (m32) {  // faces are listed in ascending id: the lowest lane is the lowest id
                    found = sc.s_tri[base + __ffs(m32) - 1];
                    break;
                }
            }
            if (found < 0) { ok = false; break; }
            face[k - 1] = found;
        }
    }
    if ((!kSolo && lane != 0) || !ok) return ok;
    o.nb_o[i] = m;
    for (int k = 0; k < kKmax; ++k) {
        o.surf_o[i * kKmax + k] = k < m ? seq[k] : -1;
        o.face_o[i * kKmax + k] = face[k];
        d3 pk = k < m ? P[k + 1] : mk3(0, 0, 0);
        st3(o.pts_o + (i * kKmax + k) * 3, pk);
    }
    o.L_o[i] = norm(img[m] - Rx);
    P[0] = Tx;
    P[m + 1] = Rx;
    angles_deg(P[1] - Tx, o.aod_o + 2 * i);
    angles_deg(P[m] - Rx, o.aoa_o + 2 * i);
    o.ray_o[i] = (uint32_t)(v & 0xffffffffull);
    o.dist_o[i] = __uint_as_float((uint32_t)(v >> 32));
    // polarimetric transfer record (see kJones in sbr_internal.cuh)
    double* J = o.jones_o + i * kJones;
    for (int k = 0; k < kJones; ++k) J[k] = 0.0;
    if (m == 0) {
        J[0] = 1.0; J[2] = 1.0; J[32] = 1.0; J[34] = 1.0;
        return true;
    }
    d3 sv_prev{}, pout_prev{};
    // unit segment directions, each computed once: the outgoing direction of
    // reflection k is the incoming one of reflection k + 1
    d3 din = unit(P[1] - P[0]);
    for (int k = 1; k <= m; ++k) {
        const d3 dout = unit(P[k + 1] - P[k]);
        double c = fabs(dot(din, nn[k]));
        d3 sv = s_vector(din, nn[k]);
        d3 pin = cross(sv, din), pout = cross(sv, dout);
        J[36 + k - 1] = c;
        if (k == 1) {
            d3 d0 = din;
            d3 eV = pol_vec(d0, SBR_POL_V), eH = pol_vec(d0, SBR_POL_H);
            J[0] = dot(eV, sv); J[1] = dot(eV, pin);
            J[2] = dot(eH, sv); J[3] = dot(eH, pin);
        } else {
            double* M = J + 4 + 4 * (k - 2);
            M[0] = dot(sv, sv_prev);  M[1] = dot(sv, pout_prev);
            M[2] = dot(pin, sv_prev); M[3] = dot(pin, pout_prev);
        }
        sv_prev = sv;
        pout_prev = pout;
        din = dout;
    }
    const d3 dl = din;   // unit(P[m + 1] - P[m])
    d3 rV = pol_vec(dl, SBR_POL_V), rH = pol_vec(dl, SBR_POL_H);
    J[32] = dot(rV, sv_prev); J[33] = dot(rV, pout_prev);
    J[34] = dot(rH, sv_prev); J[35] = dot(rH, pout_prev);
    return true;
}

}  // namespace
}  // namespace sbr
