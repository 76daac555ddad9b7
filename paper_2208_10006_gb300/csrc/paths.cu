// Effective paths (Sec. II-A.2 "pick out effective paths"; image method,
// Sec. I). The dedup table left by the trace is compacted, its keys sorted by
// (rx, n_bounce, surface sequence), and every key refined in FP64:
//   mirror the Tx through the surface planes in order (I_0 = Tx,
//   I_k = I_{k-1} - 2 (n_k.I_{k-1} - c_k) n_k), back-trace from the Rx
//   (P_m on segment I_m -> Rx, P_k on segment I_k -> P_{k+1}), require each
//   segment parameter in (0, 1) and each P_k inside one of its surface's
//   triangles (barycentric tolerance 1e-9), report the lowest-id such face,
//   and L = |I_m - Rx|.
// The plane of a surface is that of its lowest-id face. Invalid keys (ray-tube
// artefacts near edges) are dropped and counted; the rest keep key order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sbr_internal.cuh"

namespace sbr {
namespace {

constexpr int kThreads = 256;
inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

__global__ void k_collect(const uint32_t* __restrict__ state, size_t cap, uint32_t* __restrict__ idx,
                          unsigned int* __restrict__ count) {
    size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ready = s < cap && state[s] == 2u;
    unsigned m = __ballot_sync(0xffffffffu, ready);
    if (!m) return;
    unsigned base = 0;
    int lane = threadIdx.x & 31;
    if (lane == 0) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (ready) idx[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)s;
}

// sortable form of key word w of slot idx[perm[i]]: surface ids shifted by one
// so that the -1 padding sorts first
__global__ void k_key_word(const uint32_t* __restrict__ key, const uint32_t* __restrict__ idx,
                           const uint32_t* __restrict__ perm, int64_t n, int w,
                           uint32_t* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t v = key[(size_t)idx[perm[i]] * kKeyWords + w];
    out[i] = w >= 2 ? v + 1u : v;
}

__global__ void k_iota(uint32_t* p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (uint32_t)i;
}

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

// FP32 screen of the same barycentric test: +1 clearly inside, -1 clearly
// outside, 0 near an edge (then the FP64 test decides). The margin is 1e-3 or,
// for small or thin faces far from the origin, a bound on the FP32 error of
// the barycentrics (rounding of p and of the products, ~ eps (|a| + |w|) / (size sin^2)).
__device__ __forceinline__ int screen_in_tri(const float* v, float3 p) {
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
    return m > margin ? 1 : (m < -margin ? -1 : 0);
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

struct RefineArgs {
    const uint32_t* key;
    const unsigned long long* val;
    const uint32_t* idx;
    const uint32_t* perm;
    int64_t n;
    const float* tri;
    const double* nrm;
    const int32_t* s_off;
    const int32_t* s_tri;
    int32_t S;
    double tx[3];
    const double* rx;
    // raw outputs, key order
    uint32_t* valid;
    int32_t* rx_o;
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

// one warp per key: every lane runs the (cheap) image construction, the lanes
// split the containment tests over the surface's faces, lane 0 writes
__global__ void k_refine(const __grid_constant__ RefineArgs a) {
    const int lane = threadIdx.x & 31;
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= a.n) return;
    uint32_t slot = a.idx[a.perm[i]];
    const uint32_t* key = a.key + (size_t)slot * kKeyWords;
    unsigned long long v = a.val[slot];
    int rx_id = (int)key[0];
    int m = (int)key[1];
    int32_t seq[kKmax];
    for (int k = 0; k < kKmax; ++k) seq[k] = (int32_t)key[2 + k];
    d3 Tx = mk3(a.tx[0], a.tx[1], a.tx[2]);
    d3 Rx = ld3(a.rx + 3 * rx_id);
    d3 nn[kKmax + 1], img[kKmax + 1], P[kKmax + 2];
    double cc[kKmax + 1];
    bool ok = m >= 0 && m <= kKmax;
    img[0] = Tx;
    for (int k = 1; k <= m && ok; ++k) {
        int s = seq[k - 1];
        if (s < 0 || s >= a.S || a.s_off[s] == a.s_off[s + 1]) { ok = false; break; }
        int32_t t0 = a.s_tri[a.s_off[s]];
        nn[k] = ld3(a.nrm + 3 * (int64_t)t0);
        cc[k] = dot(nn[k], mk3(a.tri[9 * (int64_t)t0], a.tri[9 * (int64_t)t0 + 1], a.tri[9 * (int64_t)t0 + 2]));
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
    int32_t face[kKmax];
    for (int k = 0; k < kKmax; ++k) face[k] = -1;
    for (int k = 1; k <= m && ok; ++k) {
        int s = seq[k - 1];
        int32_t found = -1;
        const int32_t qa = a.s_off[s], qb = a.s_off[s + 1];
        for (int32_t base = qa; base < qb; base += 32) {
            int32_t q = base + lane;
            bool in = false;
            if (q < qb) {
                const float* v = a.tri + 9 * (int64_t)a.s_tri[q];
                int sc = screen_in_tri(v, make_float3((float)P[k].x, (float)P[k].y, (float)P[k].z));
                in = sc > 0 || (sc == 0 && point_in_tri(v, P[k], 1e-9));
            }
            unsigned m32 = __ballot_sync(0xffffffffu, in);
            if (m32) {  // faces are listed in ascending id: the lowest lane is the lowest id
                found = a.s_tri[base + __ffs(m32) - 1];
                break;
            }
        }
        if (found < 0) { ok = false; break; }
        face[k - 1] = found;
    }
    if (lane != 0) return;
    a.valid[i] = ok ? 1u : 0u;
    if (!ok) return;
    a.rx_o[i] = rx_id;
    a.nb_o[i] = m;
    for (int k = 0; k < kKmax; ++k) {
        a.surf_o[i * kKmax + k] = k < m ? seq[k] : -1;
        a.face_o[i * kKmax + k] = face[k];
        d3 pk = k < m ? P[k + 1] : mk3(0, 0, 0);
        st3(a.pts_o + (i * kKmax + k) * 3, pk);
    }
    a.L_o[i] = norm(img[m] - Rx);
    P[0] = Tx;
    P[m + 1] = Rx;
    angles_deg(P[1] - Tx, a.aod_o + 2 * i);
    angles_deg(P[m] - Rx, a.aoa_o + 2 * i);
    a.ray_o[i] = (uint32_t)(v & 0xffffffffull);
    a.dist_o[i] = __uint_as_float((uint32_t)(v >> 32));
    // polarimetric transfer record (see kJones in sbr_internal.cuh)
    double* J = a.jones_o + i * kJones;
    for (int k = 0; k < kJones; ++k) J[k] = 0.0;
    if (m == 0) {
        J[0] = 1.0; J[2] = 1.0; J[32] = 1.0; J[34] = 1.0;
        return;
    }
    d3 sv_prev{}, pout_prev{};
    for (int k = 1; k <= m; ++k) {
        d3 din = unit(P[k] - P[k - 1]), dout = unit(P[k + 1] - P[k]);
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
    }
    d3 dl = unit(P[m + 1] - P[m]);
    d3 rV = pol_vec(dl, SBR_POL_V), rH = pol_vec(dl, SBR_POL_H);
    J[32] = dot(rV, sv_prev); J[33] = dot(rV, pout_prev);
    J[34] = dot(rH, sv_prev); J[35] = dot(rH, pout_prev);
}

// move valid refined keys to their compacted positions: one warp per key, the
// lanes stride over the 32-bit words of all fields of the record
struct CompactArgs {
    const uint32_t* valid;
    const uint32_t* pos;
    int64_t n;
    const void* src[11];
    void* dst[11];
    int words[11];   // 32-bit words per record of each field
};

__global__ void k_compact_all(const __grid_constant__ CompactArgs a) {
    const int lane = threadIdx.x & 31;
    int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= a.n || !a.valid[r]) return;
    const int64_t q = a.pos[r];
    for (int f = 0; f < 11; ++f) {
        const uint32_t* s = static_cast<const uint32_t*>(a.src[f]) + r * a.words[f];
        uint32_t* d = static_cast<uint32_t*>(a.dst[f]) + q * a.words[f];
        for (int w = lane; w < a.words[f]; w += 32) d[w] = s[w];
    }
}

__global__ void k_rx_offsets(const int32_t* __restrict__ rx, int64_t P, int32_t n_rx,
                             int32_t* __restrict__ off) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n_rx) return;
    int64_t lo = 0, hi = P;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (rx[mid] < r) lo = mid + 1; else hi = mid;
    }
    off[r] = (int32_t)lo;
}

int bits_for(int64_t maxval) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) <= maxval) ++b;
    return b;
}

}  // namespace

sbr_status paths_run(const sbr_trace_result* tr, const sbr_bvh* b, sbr_path_list* pl, cudaStream_t s) {
    const size_t cap = (size_t)1 << tr->table_log2;
    const int K = tr->params.max_bounces;
    pl->n_rx = tr->n_rx;
    pl->K = K;
    for (int k = 0; k < 3; ++k) pl->tx[k] = tr->params.tx[k];
    SBR_TRY(dalloc_n(&pl->rx_xyz, 3 * (size_t)std::max(1, tr->n_rx), s));
    if (tr->n_rx > 0)
        SBR_TRY_CUDA(cudaMemcpyAsync(pl->rx_xyz, tr->rx, sizeof(double) * 3 * tr->n_rx,
                                     cudaMemcpyDeviceToDevice, s));
    unsigned int* count;
    uint32_t* idx;
    SBR_TRY(dalloc_n(&count, 1, s));
    SBR_TRY(dalloc_n(&idx, cap, s));
    SBR_TRY_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
    ::sbr::note_launch(), k_collect<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(tr->ht_state, cap, idx, count);
    SBR_TRY_CUDA(cudaGetLastError());
    unsigned h_count = 0;
    SBR_TRY_CUDA(cudaMemcpyAsync(&h_count, count, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SBR_TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t n = h_count;
    pl->n_keys = n;
    // sort keys: least significant word first (stable LSD over words)
    uint32_t *perm, *word;
    SBR_TRY(dalloc_n(&perm, std::max<int64_t>(n, 1), s));
    SBR_TRY(dalloc_n(&word, std::max<int64_t>(n, 1), s));
    ::sbr::note_launch(), k_iota<<<nblk(n), kThreads, 0, s>>>(perm, n);
    std::vector<std::pair<int, int>> words;  // (word index, bits)
    for (int k = K - 1; k >= 0; --k) words.push_back({2 + k, bits_for((int64_t)b->S)});
    words.push_back({1, bits_for(K)});
    words.push_back({0, bits_for(std::max(1, tr->n_rx - 1))});
    for (auto& w : words) {
        ::sbr::note_launch(), k_key_word<<<nblk(n), kThreads, 0, s>>>(tr->ht_key, idx, perm, n, w.first, word);
        SBR_TRY_CUDA(cudaGetLastError());
        SBR_TRY(radix_sort_pairs(word, perm, n, w.second, s));
    }
    // refine into raw (key-order) buffers
    RefineArgs a{};
    a.key = tr->ht_key;
    a.val = tr->ht_val;
    a.idx = idx;
    a.perm = perm;
    a.n = n;
    a.tri = b->tri;
    a.nrm = b->nrm;
    a.s_off = b->s_off;
    a.s_tri = b->s_tri;
    a.S = b->S;
    for (int k = 0; k < 3; ++k) a.tx[k] = tr->params.tx[k];
    a.rx = tr->rx;
    int64_t nn = std::max<int64_t>(n, 1);
    uint32_t* valid;
    uint32_t* pos;
    SBR_TRY(dalloc_n(&valid, nn, s));
    SBR_TRY(dalloc_n(&pos, nn, s));
    SBR_TRY(dalloc_n(&a.rx_o, nn, s));
    SBR_TRY(dalloc_n(&a.nb_o, nn, s));
    SBR_TRY(dalloc_n(&a.surf_o, nn * kKmax, s));
    SBR_TRY(dalloc_n(&a.face_o, nn * kKmax, s));
    SBR_TRY(dalloc_n(&a.pts_o, nn * kKmax * 3, s));
    SBR_TRY(dalloc_n(&a.L_o, nn, s));
    SBR_TRY(dalloc_n(&a.aod_o, nn * 2, s));
    SBR_TRY(dalloc_n(&a.aoa_o, nn * 2, s));
    SBR_TRY(dalloc_n(&a.ray_o, nn, s));
    SBR_TRY(dalloc_n(&a.dist_o, nn, s));
    SBR_TRY(dalloc_n(&a.jones_o, nn * kJones, s));
    a.valid = valid;
    if (n > 0) {
        ::sbr::note_launch(), k_refine<<<nblk(32 * n), kThreads, 0, s>>>(a);
        SBR_TRY_CUDA(cudaGetLastError());
        SBR_TRY_CUDA(cudaMemcpyAsync(pos, valid, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    SBR_TRY(exclusive_scan_u32(pos, n, count, s));
    SBR_TRY_CUDA(cudaMemcpyAsync(&h_count, count, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SBR_TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t P = h_count;
    pl->P = P;
    pl->n_invalid = n - P;
    int64_t Pp = std::max<int64_t>(P, 1);
    SBR_TRY(dalloc_n(&pl->rx, Pp, s));
    SBR_TRY(dalloc_n(&pl->nb, Pp, s));
    SBR_TRY(dalloc_n(&pl->surf, Pp * kKmax, s));
    SBR_TRY(dalloc_n(&pl->face, Pp * kKmax, s));
    SBR_TRY(dalloc_n(&pl->pts, Pp * kKmax * 3, s));
    SBR_TRY(dalloc_n(&pl->L, Pp, s));
    SBR_TRY(dalloc_n(&pl->aod, Pp * 2, s));
    SBR_TRY(dalloc_n(&pl->aoa, Pp * 2, s));
    SBR_TRY(dalloc_n(&pl->ray, Pp, s));
    SBR_TRY(dalloc_n(&pl->dist, Pp, s));
    SBR_TRY(dalloc_n(&pl->jones, Pp * kJones, s));
    SBR_TRY(dalloc_n(&pl->rx_off, (size_t)tr->n_rx + 1, s));
    SBR_TRY(dalloc_n(&pl->d_status, 1, s));
    SBR_TRY_CUDA(cudaMemsetAsync(pl->d_status, 0, sizeof(unsigned), s));
    if (n > 0) {
        CompactArgs c{};
        c.valid = valid;
        c.pos = pos;
        c.n = n;
        const void* src[11] = {a.rx_o, a.nb_o, a.surf_o, a.face_o, a.pts_o, a.L_o, a.aod_o, a.aoa_o,
                               a.ray_o, a.dist_o, a.jones_o};
        void* dst[11] = {pl->rx, pl->nb, pl->surf, pl->face, pl->pts, pl->L, pl->aod, pl->aoa, pl->ray,
                         pl->dist, pl->jones};
        const int words[11] = {1, 1, kKmax, kKmax, 2 * 3 * kKmax, 2, 4, 4, 1, 1, 2 * kJones};
        for (int f = 0; f < 11; ++f) { c.src[f] = src[f]; c.dst[f] = dst[f]; c.words[f] = words[f]; }
        ::sbr::note_launch(), k_compact_all<<<nblk(32 * n), kThreads, 0, s>>>(c);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    ::sbr::note_launch(), k_rx_offsets<<<nblk((int64_t)tr->n_rx + 1), kThreads, 0, s>>>(pl->rx, P, tr->n_rx, pl->rx_off);
    SBR_TRY_CUDA(cudaGetLastError());
    pl->h_rx_off = new int32_t[tr->n_rx + 1];
    SBR_TRY_CUDA(cudaMemcpyAsync(pl->h_rx_off, pl->rx_off, sizeof(int32_t) * (tr->n_rx + 1),
                                 cudaMemcpyDeviceToHost, s));
    SBR_TRY_CUDA(cudaStreamSynchronize(s));
    dfree(count, s); dfree(idx, s); dfree(perm, s); dfree(word, s); dfree(valid, s); dfree(pos, s);
    dfree(a.rx_o, s); dfree(a.nb_o, s); dfree(a.surf_o, s); dfree(a.face_o, s); dfree(a.pts_o, s);
    dfree(a.L_o, s); dfree(a.aod_o, s); dfree(a.aoa_o, s); dfree(a.ray_o, s); dfree(a.dist_o, s);
    dfree(a.jones_o, s);
    return SBR_OK;
}

}  // namespace sbr
