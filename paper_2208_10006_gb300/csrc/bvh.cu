// Acceleration structure for the intersection search (the paper parallelises
// this step on the GPU, Sec. III-C, without describing a structure).
//
// Linear BVH built entirely on the device: Morton codes of primitive
// centroids, stable radix sort, Karras radix tree (one thread per internal
// node), bottom-up box refit with atomic arrival flags, then emission into
// 64-byte nodes that hold both child boxes, so a traversal step reads one
// node and tests two boxes. Boxes are padded outward by a relative margin so
// that FP32 traversal never culls a box that the exact ray touches.
#include <algorithm>
#include <cuda/atomic>
#include <cstdlib>

#include "dfloat.cuh"
#include "sbr_internal.cuh"

namespace sbr {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int t = kThreads) {
    return (unsigned)std::max<int64_t>(1, (n + t - 1) / t);
}

// out[0..5] centroid lo/hi, out[6..11] box lo/hi (one block)
// scene bounds of the box centres (for the Morton grid) and of the boxes:
// out[0..2] centre min, [3..5] centre max, [6..8] box min, [9..11] box max.
// Stage 1: per-block partial reductions (grid-stride); stage 2: one block
// combines the partials.
__device__ __forceinline__ void bounds_block_reduce(float* v, float (*red)[32], float* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 12; ++k) {
        float x = v[k];
        bool mx = (k / 3) & 1;
        for (int o = 16; o; o >>= 1) {
            float y = __shfl_xor_sync(0xffffffffu, x, o);
            x = mx ? fmaxf(x, y) : fminf(x, y);
        }
        if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        int k = threadIdx.x;
        bool mx = (k / 3) & 1;
        float x = red[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = mx ? fmaxf(x, red[k][w]) : fminf(x, red[k][w]);
        out[k] = x;
    }
}

__global__ void k_bounds(const float* __restrict__ box, int64_t n, float* __restrict__ part) {
    ::sbr::pdl_wait();
    __shared__ float red[12][32];
    float v[12];
    for (int a = 0; a < 3; ++a) {
        v[a] = INFINITY; v[3 + a] = -INFINITY; v[6 + a] = INFINITY; v[9 + a] = -INFINITY;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            float lo = box[6 * i + a], hi = box[6 * i + 3 + a];
            float c = 0.5f * (lo + hi);
            v[a] = fminf(v[a], c); v[3 + a] = fmaxf(v[3 + a], c);
            v[6 + a] = fminf(v[6 + a], lo); v[9 + a] = fmaxf(v[9 + a], hi);
        }
    }
    bounds_block_reduce(v, red, part + 12 * blockIdx.x);
}

__global__ void k_bounds_final(const float* __restrict__ part, int nparts, float* __restrict__ out) {
    ::sbr::pdl_wait();
    __shared__ float red[12][32];
    float v[12];
    for (int a = 0; a < 3; ++a) {
        v[a] = INFINITY; v[3 + a] = -INFINITY; v[6 + a] = INFINITY; v[9 + a] = -INFINITY;
    }
    for (int p = threadIdx.x; p < nparts; p += blockDim.x)
        for (int k = 0; k < 12; ++k) v[k] = ((k / 3) & 1) ? fmaxf(v[k], part[12 * p + k]) : fminf(v[k], part[12 * p + k]);
    bounds_block_reduce(v, red, out);
}

// 10-bit integer spread to every third bit (the Morton interleave)
__device__ __forceinline__ uint32_t expand_bits(uint32_t x) {
    x = (x * 0x00010001u) & 0xFF0000FFu;
    x = (x * 0x00000101u) & 0x0F00F00Fu;
    x = (x * 0x00000011u) & 0xC30C30C3u;
    x = (x * 0x00000005u) & 0x49249249u;
    return x;
}

// Also clears the refit's arrival flags (nn of them, nn <= n) and the depth.
__global__ void k_morton(const float* __restrict__ box, int64_t n, const float* __restrict__ bnd,
                         uint32_t* __restrict__ code, uint32_t* __restrict__ idx, int32_t* __restrict__ flag,
                         int64_t nn, int32_t* __restrict__ depth) {
    ::sbr::pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i < nn) flag[i] = 0;
    if (i == 0) *depth = 0;
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        float c = 0.5f * (box[6 * i + a] + box[6 * i + 3 + a]);
        float ext = bnd[3 + a] - bnd[a];
        float u = ext > 0.f ? (c - bnd[a]) / ext : 0.f;
        u = fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
        q[a] = (uint32_t)u;
    }
    code[i] = (expand_bits(q[0]) << 2) | (expand_bits(q[1]) << 1) | expand_bits(q[2]);
    idx[i] = (uint32_t)i;
}

// longest common prefix of the (code, index) keys of sorted positions i and j
__device__ __forceinline__ int delta(const uint32_t* __restrict__ code, int64_t n, int64_t i,
                                     int64_t j) {
    if (j < 0 || j >= n) return -1;
    uint64_t a = ((uint64_t)code[i] << 32) | (uint64_t)(uint32_t)i;
    uint64_t b = ((uint64_t)code[j] << 32) | (uint64_t)(uint32_t)j;
    return __clzll((long long)(a ^ b));
}

__global__ void k_karras(const uint32_t* __restrict__ code, int64_t n, int32_t* __restrict__ left,
                         int32_t* __restrict__ right, int32_t* __restrict__ parent_int,
                         int32_t* __restrict__ parent_leaf, int32_t* __restrict__ span) {
    ::sbr::pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(code, n, i, i + 1) - delta(code, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(code, n, i, i - d);
    int64_t lmax = 2;
    while (delta(code, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(code, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(code, n, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(code, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    span[2 * i] = (int32_t)lo;       // the node covers sorted primitives [lo, hi]
    span[2 * i + 1] = (int32_t)hi;
    if (lo == gamma) {
        left[i] = ~(int32_t)gamma;
        parent_leaf[gamma] = (int32_t)i;
    } else {
        left[i] = (int32_t)gamma;
        parent_int[gamma] = (int32_t)i;
    }
    if (hi == gamma + 1) {
        right[i] = ~(int32_t)(gamma + 1);
        parent_leaf[gamma + 1] = (int32_t)i;
    } else {
        right[i] = (int32_t)(gamma + 1);
        parent_int[gamma + 1] = (int32_t)i;
    }
    if (i == 0) parent_int[0] = -1;
}

__device__ __forceinline__ void ld_box(const float* p, float b[6]) {
    const volatile float* q = p;
    for (int k = 0; k < 6; ++k) b[k] = q[k];
}

__global__ void k_refit(const float* __restrict__ prim_box, const int32_t* __restrict__ order,
                        int64_t n, const int32_t* __restrict__ left,
                        const int32_t* __restrict__ right, const int32_t* __restrict__ parent_int,
                        const int32_t* __restrict__ parent_leaf, int32_t* __restrict__ flag,
                        float* lbox, float* ibox, int32_t* hd, int32_t* __restrict__ depth) {
    ::sbr::pdl_wait();
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float* src = prim_box + 6 * (int64_t)order[j];
    for (int k = 0; k < 6; ++k) lbox[6 * j + k] = src[k];
    if (n < 2) {
        *depth = 1;
        return;
    }
    // the climbing thread carries its subtree's box and height and reads only
    // the sibling's; the node's children and parent (read-only here) are
    // fetched before the arrival count, so each level costs the count and one
    // dependent load
    float a[6];
    for (int k = 0; k < 6; ++k) a[k] = src[k];
    int32_t me = ~(int32_t)j, h = 1;
    int32_t node = parent_leaf[j];
    while (node >= 0) {
        const int32_t l = left[node], r = right[node], up = parent_int[node];
        // release: this thread's boxes before the count; acquire: the sibling's after it
        cuda::atomic_ref<int32_t, cuda::thread_scope_device> cnt(flag[node]);
        if (cnt.fetch_add(1, cuda::memory_order_acq_rel) == 0) return;  // the sibling subtree is not done yet
        const int32_t sib = l == me ? r : l;
        float b[6];
        ld_box(sib < 0 ? lbox + 6 * (int64_t)(~sib) : ibox + 6 * (int64_t)sib, b);
        // height: a leaf counts 1, a node one more than its higher child; the
        // root's height is the tree depth (levels on the longest root-leaf path)
        const int hs = sib < 0 ? 1 : ((volatile int32_t*)hd)[sib];
        volatile float* o = ibox + 6 * (int64_t)node;
        for (int k = 0; k < 3; ++k) {
            a[k] = fminf(a[k], b[k]);
            a[3 + k] = fmaxf(a[3 + k], b[3 + k]);
            o[k] = a[k];
            o[3 + k] = a[3 + k];
        }
        h = 1 + (h > hs ? h : hs);
        ((volatile int32_t*)hd)[node] = h;
        if (up < 0) *depth = h;
        me = node;
        node = up;
    }
}

__device__ __forceinline__ float pad_lo(float x, float pad) { return x - pad * (fabsf(x) + 1.f); }
__device__ __forceinline__ float pad_hi(float x, float pad) { return x + pad * (fabsf(x) + 1.f); }

// child reference: internal node index, or a leaf ~(first | (count - 1) << 28)
// holding `count` consecutive sorted primitives; subtrees of at most leaf_max
// primitives are emitted as one leaf (their primitives are consecutive in
// Morton order), so traversal stops above them
__device__ __forceinline__ int32_t child_ref(int32_t c, const int32_t* __restrict__ span, int leaf_max) {
    if (c < 0) return c;  // single primitive ~p (count 1)
    int32_t lo = span[2 * c], hi = span[2 * c + 1];
    if (hi - lo + 1 <= leaf_max) return ~(lo | ((hi - lo) << 28));
    return c;
}

__global__ void k_emit(int64_t n, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                       const int32_t* __restrict__ span, int leaf_max,
                       const float* __restrict__ lbox, const float* __restrict__ ibox, float pad,
                       float4* __restrict__ nodes, float* __restrict__ root) {
    ::sbr::pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nn = n > 1 ? n - 1 : 1;
    if (i >= nn) return;
    float b0[6], b1[6];
    int32_t r0, r1;
    if (n == 1) {
        // single primitive: both children name leaf 0. The FP32 closest-hit
        // traversal then tests that leaf twice, which changes nothing (a repeated
        // face neither improves the best hit nor enters the uncertain list
        // twice); the other traversals skip r1 == r0
        for (int k = 0; k < 6; ++k) b0[k] = b1[k] = lbox[k];
        r0 = ~0; r1 = ~0;
    } else {
        r0 = left[i]; r1 = right[i];
        const float* p0 = r0 < 0 ? lbox + 6 * (int64_t)(~r0) : ibox + 6 * (int64_t)r0;
        const float* p1 = r1 < 0 ? lbox + 6 * (int64_t)(~r1) : ibox + 6 * (int64_t)r1;
        for (int k = 0; k < 6; ++k) { b0[k] = p0[k]; b1[k] = p1[k]; }
        r0 = child_ref(r0, span, leaf_max);
        r1 = child_ref(r1, span, leaf_max);
    }
    for (int k = 0; k < 3; ++k) {
        b0[k] = pad_lo(b0[k], pad); b0[3 + k] = pad_hi(b0[3 + k], pad);
        b1[k] = pad_lo(b1[k], pad); b1[3 + k] = pad_hi(b1[3 + k], pad);
    }
    float4* o = nodes + 4 * i;
    o[0] = make_float4(b0[0], b0[1], b0[2], b0[3]);
    o[1] = make_float4(b0[4], b0[5], b1[0], b1[1]);
    o[2] = make_float4(b1[2], b1[3], b1[4], b1[5]);
    o[3] = make_float4(__int_as_float(r0), __int_as_float(r1), 0.f, 0.f);
    if (i == 0) {
        const float* rb = n > 1 ? ibox : lbox;
        for (int k = 0; k < 3; ++k) { root[k] = pad_lo(rb[k], pad); root[3 + k] = pad_hi(rb[3 + k], pad); }
    }
}

// ---------------------------------------------------------------- SAH top levels
// The Morton order places the first splits of the tree by position on the
// space-filling curve, not by cost. The top of the tree is rebuilt with the
// surface-area heuristic: the subtrees of at most `lim` primitives hanging
// below it (the cut) become the items of a top-down binned SAH build (32 bins
// per axis over the item centroids), which reuses the node slots of the old
// top (a binary tree over C items has C - 1 nodes, and the root stays node 0).
// The items' boxes are the padded child boxes of their old parents, so the new
// boxes stay conservative. The cut holds about 650 subtrees (lim = n / 400):
// on the urban scene (51,600 triangles) a cut of 1,300 subtrees gives 6.7%
// fewer node visits per segment than the Morton top, one of 300 gives 6%, a
// full SAH build 11%. Each warp gathers its bins lane by lane over all of a
// task's items, so the top levels are serial: the build takes 0.2-1.2 ms.
struct TopElem {
    float b[6];
    int32_t ref;
    int32_t h;      // height of the subtree (levels)
};
struct TopTask {
    int32_t begin, count, slot, depth;
};
constexpr int kTopCap = 2048;      // items at most (held in shared memory; else the Morton top is kept)
constexpr int kTopWarps = 16;
constexpr int kTopBins = 32;
constexpr int kTopForceMedian = 48;   // depth from which splits are by position (ends the build)
constexpr int kTopMaxLevels = 96;

__device__ __forceinline__ int span_size(const int32_t* span, int32_t r) {
    return r < 0 ? leaf_count(r) : span[2 * r + 1] - span[2 * r] + 1;
}

// the cut: children of size <= lim of the nodes of size > lim; the slots of
// those nodes (node 0 excepted) are reused for the new top
__global__ void k_top_cut(int64_t nn, const int32_t* __restrict__ span, const int32_t* __restrict__ hd,
                          const float4* __restrict__ nodes, int lim, TopElem* __restrict__ E, int* n_cut,
                          int32_t* __restrict__ slots, int* n_slot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn || span_size(span, (int32_t)i) <= lim) return;
    if (i != 0) {
        const int k = atomicAdd(n_slot, 1);
        if (k < kTopCap) slots[k] = (int32_t)i;
    }
    const float4* nd = nodes + 4 * i;
    const float4 n0 = nd[0], n1 = nd[1], n2 = nd[2], n3 = nd[3];
    const int32_t r[2] = {__float_as_int(n3.x), __float_as_int(n3.y)};
    const float bx[2][6] = {{n0.x, n0.y, n0.z, n0.w, n1.x, n1.y}, {n1.z, n1.w, n2.x, n2.y, n2.z, n2.w}};
    for (int c = 0; c < 2; ++c) {
        if (span_size(span, r[c]) > lim) continue;
        const int e = atomicAdd(n_cut, 1);
        if (e >= kTopCap) continue;
        TopElem t;
        for (int k = 0; k < 6; ++k) t.b[k] = bx[c][k];
        t.ref = r[c];
        t.h = r[c] < 0 ? 1 : hd[r[c]];
        E[e] = t;
    }
}

__device__ __forceinline__ float box_area(const float* b) {
    const float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return 2.f * (dx * dy + dy * dz + dz * dx);
}

// warp scan of per-bin (count, box) over the 32 bins held one per lane:
// inclusive from bin 0 up (up) or from bin 31 down (!up)
__device__ __forceinline__ void bin_scan(int& c, float* b, bool up) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        const bool take = up ? lane >= o : lane + o < 32;
        const int oc = up ? __shfl_up_sync(FULL, c, o) : __shfl_down_sync(FULL, c, o);
        float ob[6];
        for (int q = 0; q < 6; ++q) ob[q] = up ? __shfl_up_sync(FULL, b[q], o) : __shfl_down_sync(FULL, b[q], o);
        if (take) {
            c += oc;
            for (int q = 0; q < 3; ++q) { b[q] = fminf(b[q], ob[q]); b[3 + q] = fmaxf(b[3 + q], ob[3 + q]); }
        }
    }
}

// lane 0 of a task's warp: the node with its two child boxes, and either the
// item (a child of one item) or a new task per child
__device__ void top_emit(const TopTask& tk, int nl, const float* sl, const float* sr, const TopElem* out,
                         float4* __restrict__ nodes, const int32_t* __restrict__ slots, TopTask* next, int* s_next,
                         int* s_slot, int* s_depth) {
    const int b0 = tk.begin, n = tk.count;
    int32_t ref[2];
    const int cb[2] = {b0, b0 + nl}, cn[2] = {nl, n - nl};
    for (int c = 0; c < 2; ++c) {
        if (cn[c] == 1) {
            ref[c] = out[cb[c]].ref;
            atomicMax(s_depth, tk.depth + out[cb[c]].h);
        } else {
            ref[c] = slots[atomicAdd(s_slot, 1)];
            next[atomicAdd(s_next, 1)] = TopTask{cb[c], cn[c], ref[c], tk.depth + 1};
        }
    }
    float4* o = nodes + 4 * (int64_t)tk.slot;
    o[0] = make_float4(sl[0], sl[1], sl[2], sl[3]);
    o[1] = make_float4(sl[4], sl[5], sr[0], sr[1]);
    o[2] = make_float4(sr[2], sr[3], sr[4], sr[5]);
    o[3] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), 0.f, 0.f);
}

// float <-> int with the same order (for shared-memory atomicMin / atomicMax
// on box bounds): the magnitude bits of a negative value are flipped
__device__ __forceinline__ int ord_f(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unord_f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }
constexpr int kTopBinWords = 3 * kTopBins * 7;   // per warp: count and 6 bounds of every bin of each axis

// one warp: split one task, write its node, queue its children. The items sit
// in shared memory; the lanes bin the task's items in parallel into the warp's
// shared-memory bins (counts by atomicAdd, bounds by atomicMin / atomicMax on
// order-preserving integers: exact, so the split is independent of the
// order), lane b then takes bin b of each axis, and warp scans give every
// split's two sides.
__device__ void top_task(const TopTask tk, const TopElem* in, TopElem* out, float4* __restrict__ nodes,
                         const int32_t* __restrict__ slots, TopTask* next, int* s_next, int* s_slot, int* s_depth,
                         int* wbins) {
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int b0 = tk.begin, n = tk.count;
    // centroid bounds
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = lane; i < n; i += 32)
        for (int a = 0; a < 3; ++a) {
            const float c = 0.5f * (in[b0 + i].b[a] + in[b0 + i].b[3 + a]);
            lo[a] = fminf(lo[a], c);
            hi[a] = fmaxf(hi[a], c);
        }
    for (int o = 16; o; o >>= 1)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(FULL, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(FULL, hi[a], o));
        }
    float sc[3];
    for (int a = 0; a < 3; ++a) sc[a] = hi[a] > lo[a] ? (float)kTopBins / (hi[a] - lo[a]) : 0.f;
    // bin the items: wbins[a][b] = count, then [a][b][6] bounds
    int* const bcnt = wbins;
    int* const bbox = wbins + 3 * kTopBins;
    for (int j = lane; j < 3 * kTopBins; j += 32) bcnt[j] = 0;
    for (int j = lane; j < 3 * kTopBins * 6; j += 32) bbox[j] = ord_f(j % 6 < 3 ? INFINITY : -INFINITY);
    __syncwarp();
    // each lane takes a contiguous segment of the items: the items are in
    // Morton order, so the 32 items of one round lie far apart and mostly
    // update different bins
    const int per = (n + 31) / 32;
    for (int k = 0; k < per; ++k) {
        const int i = lane * per + k;
        if (i >= n) break;
        const TopElem& e = in[b0 + i];
        for (int a = 0; a < 3; ++a) {
            if (sc[a] == 0.f) continue;
            const int bin = min(kTopBins - 1, (int)((0.5f * (e.b[a] + e.b[3 + a]) - lo[a]) * sc[a]));
            atomicAdd(&bcnt[a * kTopBins + bin], 1);
            int* bb = bbox + (a * kTopBins + bin) * 6;
            for (int q = 0; q < 3; ++q) {
                atomicMin(&bb[q], ord_f(e.b[q]));
                atomicMax(&bb[3 + q], ord_f(e.b[3 + q]));
            }
        }
    }
    __syncwarp();
    // this lane's bin (number lane) of each axis
    int cnt[3];
    float bx[3][6];
    for (int a = 0; a < 3; ++a) {
        cnt[a] = bcnt[a * kTopBins + lane];
        for (int q = 0; q < 6; ++q) bx[a][q] = unord_f(bbox[(a * kTopBins + lane) * 6 + q]);
    }
    __syncwarp();   // the bins are rewritten by this warp's next task
    // split "bins below s go left" with s = lane (1..31): left = prefix through bin s-1, right =
    // suffix from bin s; each lane keeps its best axis with the counts and boxes of both sides
    float best = INFINITY;
    int bcode = 0x7fffffff, bnl = 0;
    float bl[6], br[6];
    for (int a = 0; a < 3; ++a) {
        int cp = cnt[a], cs = cnt[a];
        float pb[6], sb6[6];
        for (int q = 0; q < 6; ++q) { pb[q] = bx[a][q]; sb6[q] = bx[a][q]; }
        bin_scan(cp, pb, true);
        bin_scan(cs, sb6, false);
        // the prefix through bin lane - 1 comes from the lane below
        const int nl = __shfl_up_sync(FULL, cp, 1);
        float L[6];
        for (int q = 0; q < 6; ++q) L[q] = __shfl_up_sync(FULL, pb[q], 1);
        if (lane == 0 || sc[a] == 0.f || tk.depth >= kTopForceMedian || nl == 0 || cs == 0) continue;
        const float cost = box_area(L) * nl + box_area(sb6) * cs;
        const int code = a * kTopBins + lane;
        if (cost < best || (cost == best && code < bcode)) {
            best = cost; bcode = code; bnl = nl;
            for (int q = 0; q < 6; ++q) { bl[q] = L[q]; br[q] = sb6[q]; }
        }
    }
    // the warp's best split (ties to the lowest axis, then the lowest s)
    float wb = best;
    int wc = bcode;
    for (int o = 16; o; o >>= 1) {
        const float ob = __shfl_xor_sync(FULL, wb, o);
        const int oc = __shfl_xor_sync(FULL, wc, o);
        if (ob < wb || (ob == wb && oc < wc)) { wb = ob; wc = oc; }
    }
    const bool by_pos = !(wb < INFINITY);   // no split with both sides non-empty: split by position
    const int ax = by_pos ? 0 : wc / kTopBins, sb = by_pos ? 0 : wc % kTopBins;
    const int nl = by_pos ? n / 2 : __shfl_sync(FULL, bnl, sb);
    float sl[6], sr[6];
    for (int q = 0; q < 6; ++q) {
        sl[q] = __shfl_sync(FULL, bl[q], by_pos ? 0 : sb);
        sr[q] = __shfl_sync(FULL, br[q], by_pos ? 0 : sb);
    }
    // stable partition into out[b0, b0 + n)
    int cl = 0, cr = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        bool left = false;
        TopElem e;
        if (i < n) {
            e = in[b0 + i];
            if (by_pos) {
                left = i < nl;
            } else {
                const int bin = min(kTopBins - 1, (int)((0.5f * (e.b[ax] + e.b[3 + ax]) - lo[ax]) * sc[ax]));
                left = bin < sb;
            }
        }
        const unsigned ml = __ballot_sync(FULL, i < n && left), mr = __ballot_sync(FULL, i < n && !left);
        const unsigned lt = (1u << lane) - 1u;
        if (i < n) out[b0 + (left ? cl + __popc(ml & lt) : nl + cr + __popc(mr & lt))] = e;
        cl += __popc(ml);
        cr += __popc(mr);
    }
    __syncwarp();
    if (by_pos) {   // side boxes by reduction over the two halves
        for (int q = 0; q < 3; ++q) { sl[q] = INFINITY; sl[3 + q] = -INFINITY; sr[q] = INFINITY; sr[3 + q] = -INFINITY; }
        for (int i = lane; i < n; i += 32) {
            float* D = i < nl ? sl : sr;
            const TopElem& e = out[b0 + i];
            for (int q = 0; q < 3; ++q) { D[q] = fminf(D[q], e.b[q]); D[3 + q] = fmaxf(D[3 + q], e.b[3 + q]); }
        }
        for (int o = 16; o; o >>= 1)
            for (int q = 0; q < 3; ++q) {
                sl[q] = fminf(sl[q], __shfl_xor_sync(FULL, sl[q], o));
                sl[3 + q] = fmaxf(sl[3 + q], __shfl_xor_sync(FULL, sl[3 + q], o));
                sr[q] = fminf(sr[q], __shfl_xor_sync(FULL, sr[q], o));
                sr[3 + q] = fmaxf(sr[3 + q], __shfl_xor_sync(FULL, sr[3 + q], o));
            }
    }
    if (lane == 0) top_emit(tk, nl, sl, sr, out, nodes, slots, next, s_next, s_slot, s_depth);
    __syncwarp();
}

// one block: the top tree over the cut, level by level (the tasks of a level
// are independent: disjoint item ranges, distinct node slots); items and task
// lists in shared memory
constexpr int kTopSmem = 2 * kTopCap * (int)sizeof(TopElem) + 2 * (kTopCap / 2 + 1) * (int)sizeof(TopTask) +
                         kTopWarps * kTopBinWords * (int)sizeof(int);

__global__ void __launch_bounds__(32 * kTopWarps)
k_top_sah(float4* __restrict__ nodes, const TopElem* __restrict__ E, const int32_t* __restrict__ slots,
          const int* n_cut, const int* n_slot, int32_t* d_depth) {
    extern __shared__ unsigned char s_top[];
    TopElem* S0 = reinterpret_cast<TopElem*>(s_top);
    TopElem* S1 = S0 + kTopCap;
    TopTask* Q0 = reinterpret_cast<TopTask*>(S1 + kTopCap);
    TopTask* Q1 = Q0 + kTopCap / 2 + 1;
    int* bins = reinterpret_cast<int*>(Q1 + kTopCap / 2 + 1);   // [kTopWarps][kTopBinWords]
    __shared__ int s_nt, s_next, s_slot, s_depth;
    const int warp = threadIdx.x >> 5;
    const int C = *n_cut;
    // a cut of C items hangs below C - 1 old nodes: the root and C - 2 reusable slots
    if (C < 2 || C > kTopCap || *n_slot != C - 2) return;
    for (int i = threadIdx.x; i < C; i += blockDim.x) S0[i] = E[i];
    if (threadIdx.x == 0) {
        Q0[0] = TopTask{0, C, 0, 1};
        s_nt = 1; s_next = 0; s_slot = 0; s_depth = 0;
    }
    __syncthreads();
    TopElem *in = S0, *out = S1;
    TopTask *tin = Q0, *tout = Q1;
    for (int level = 0; level < kTopMaxLevels; ++level) {
        const int nt = s_nt;
        if (nt == 0) break;
        for (int t = warp; t < nt; t += kTopWarps)
            top_task(tin[t], in, out, nodes, slots, tout, &s_next, &s_slot, &s_depth, bins + warp * kTopBinWords);
        __syncthreads();
        if (threadIdx.x == 0) { s_nt = s_next; s_next = 0; }
        __syncthreads();
        TopElem* te = in; in = out; out = te;
        TopTask* tt = tin; tin = tout; tout = tt;
    }
    if (threadIdx.x == 0) *d_depth = s_depth;
}

// ---------------------------------------------------------------- triangles
// per face: bounding box, FP64 unit normal, and the (surface id, face id)
// pair of the faces-per-surface sort; degenerate faces and surface ids out of
// range set the status word
// The BVH's own copies of the vertices and surface ids, and per face its box,
// unit normal and surface sort key; a degenerate face or an out-of-range
// surface id sets the host-mapped word h_status.
__global__ void k_tri_prep(const float* __restrict__ tri_in, const int32_t* __restrict__ surf_in, int64_t T,
                           int32_t S, float* __restrict__ tri, int32_t* __restrict__ surf,
                           float* __restrict__ box, double* __restrict__ nrm, uint32_t* __restrict__ key,
                           uint32_t* __restrict__ val, unsigned int* h_status) {
    ::sbr::pdl_wait();
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    float v[9];
    for (int k = 0; k < 9; ++k) {
        v[k] = tri_in[9 * t + k];
        tri[9 * t + k] = v[k];
    }
    for (int a = 0; a < 3; ++a) {
        box[6 * t + a] = fminf(v[a], fminf(v[3 + a], v[6 + a]));
        box[6 * t + 3 + a] = fmaxf(v[a], fmaxf(v[3 + a], v[6 + a]));
    }
    d3 v0 = mk3(v[0], v[1], v[2]), v1 = mk3(v[3], v[4], v[5]), v2 = mk3(v[6], v[7], v[8]);
    d3 c = cross(v1 - v0, v2 - v0);
    double l = norm(c);
    bool bad = !(l > 0.0) || !isfinite(l);
    st3(nrm + 3 * t, c * (1.0 / l));
    int32_t s = surf_in[t];
    surf[t] = s;
    bad |= s < 0 || s >= S;
    if (bad) *(volatile unsigned int*)h_status = (unsigned)ST_NUMERIC;
    key[t] = (uint32_t)min(max(s, 0), S - 1);
    val[t] = (uint32_t)t;
}

// A pinned, device-mapped host word and an event per thread and device: the
// validation kernel writes its verdict straight to the host while the rest of
// the build runs, and the call waits for the validation kernel only.
struct HostFlag {
    unsigned* h = nullptr;
    unsigned* d = nullptr;   // the same word, device view
    cudaEvent_t ev = nullptr;
};

sbr_status host_flag(HostFlag** out) {
    constexpr int kMaxDev = 64;
    thread_local HostFlag flags[kMaxDev];
    int dev = 0;
    SBR_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) {
        set_error("device index %d out of range", dev);
        return SBR_ERR_UNSUPPORTED;
    }
    HostFlag& f = flags[dev];
    if (!f.h) {
        SBR_TRY_CUDA(cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming));
        SBR_TRY_CUDA(cudaHostAlloc(&f.h, sizeof(unsigned), cudaHostAllocMapped));
        SBR_TRY_CUDA(cudaHostGetDevicePointer(&f.d, f.h, 0));
    }
    *out = &f;
    return SBR_OK;
}

// The faces in BVH order, three times: block kz holds each vertex with its
// components rotated to (kz+1, kz+2, kz) mod 3, so that a ray whose dominant
// direction axis is kz reads its shear frame's coordinates without selects;
// block 2 is the plain order. w: surface id bits (v0), face id bits (v1).
__global__ void k_tri_pack(const float* __restrict__ tri, const int32_t* __restrict__ surf,
                           const double* __restrict__ nrm, const int32_t* __restrict__ order,
                           int64_t T, float4* __restrict__ rot, float4* __restrict__ plane) {
    ::sbr::pdl_wait();
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= T) return;
    int64_t t = order[j];
    const float* v = tri + 9 * t;
    const float ws = __int_as_float(surf[t]), wf = __int_as_float((int)t);
    for (int kz = 0; kz < 3; ++kz) {
        const int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
        float4* out = rot + 3 * T * kz;
        out[3 * j + 0] = make_float4(v[kx], v[ky], v[kz], ws);
        out[3 * j + 1] = make_float4(v[3 + kx], v[3 + ky], v[3 + kz], wf);
        out[3 * j + 2] = make_float4(v[6 + kx], v[6 + ky], v[6 + kz], 0.f);
    }
    // plane n.x = c with the FP64 unit normal, stored as double-float pairs
    double n0 = nrm[3 * t], n1 = nrm[3 * t + 1], n2 = nrm[3 * t + 2];
    double c = n0 * (double)v[0] + n1 * (double)v[1] + n2 * (double)v[2];
    df a = df_from_double(n0), bb = df_from_double(n1), cc = df_from_double(n2), dd = df_from_double(c);
    plane[2 * j] = make_float4(a.hi, bb.hi, cc.hi, dd.hi);
    plane[2 * j + 1] = make_float4(a.lo, bb.lo, cc.lo, dd.lo);
}

__global__ void k_surface_offsets(const uint32_t* __restrict__ key, int64_t T, int32_t S,
                                  int32_t* __restrict__ s_off) {
    ::sbr::pdl_wait();
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > S) return;
    int64_t lo = 0, hi = T;  // first position with key >= s
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (key[mid] < (uint32_t)s) lo = mid + 1; else hi = mid;
    }
    s_off[s] = (int32_t)lo;
}

}  // namespace

sbr_status build_lbvh(const float* prim_box, int64_t n, float pad_rel, int leaf_max, BvhNodes* out,
                      int32_t* d_depth, cudaStream_t s, bool top_sah) {
    *out = BvhNodes{};
    if (n <= 0) return SBR_OK;
    if (n >= (int64_t)1 << 31) {
        set_error("too many primitives for the BVH");
        return SBR_ERR_UNSUPPORTED;
    }
    int64_t nn = n > 1 ? n - 1 : 1;
    float* bnd;
    uint32_t *code, *idx;
    int32_t *left, *right, *pint, *pleaf, *flag, *span;
    float *lbox, *ibox;
    SBR_TRY(dalloc_n(&bnd, 12, s));
    float* part;
    SBR_TRY(dalloc_n(&part, 12 * 2 * (size_t)sm_count(), s));
    int32_t* hd;
    SBR_TRY(dalloc_n(&hd, nn, s));
    SBR_TRY(dalloc_n(&code, n, s));
    SBR_TRY(dalloc_n(&idx, n, s));
    SBR_TRY(dalloc_n(&left, nn, s));
    SBR_TRY(dalloc_n(&right, nn, s));
    SBR_TRY(dalloc_n(&pint, nn, s));
    SBR_TRY(dalloc_n(&pleaf, n, s));
    SBR_TRY(dalloc_n(&flag, nn, s));
    SBR_TRY(dalloc_n(&span, 2 * nn, s));
    SBR_TRY(dalloc_n(&lbox, 6 * n, s));
    SBR_TRY(dalloc_n(&ibox, 6 * nn, s));
    SBR_TRY(dalloc_n(&out->nodes, 4 * nn, s));
    SBR_TRY(dalloc_n(&out->d_root, 6, s));
    const int nparts = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 2 * (int64_t)sm_count());
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_bounds, dim3(nparts), dim3(256), 0, s, prim_box, n, part);
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_bounds_final, dim3(1), dim3(256), 0, s, part, nparts, bnd);
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_morton, dim3(blocks_for(n)), dim3(kThreads), 0, s, prim_box, n, bnd, code, idx, flag, nn, d_depth);
    SBR_TRY_CUDA(cudaGetLastError());
    SBR_TRY(radix_sort_pairs(code, idx, n, 30, s));
    if (n > 1) ::sbr::note_launch(), (void)::sbr::launch_pdl(k_karras, dim3(blocks_for(n - 1)), dim3(kThreads), 0, s, code, n, left, right, pint, pleaf, span);
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_refit, dim3(blocks_for(n)), dim3(kThreads), 0, s, prim_box, (const int32_t*)idx, n, left, right, pint,
                                               pleaf, flag, lbox, ibox, hd, d_depth);
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_emit, dim3(blocks_for(nn)), dim3(kThreads), 0, s, n, left, right, span, leaf_max, lbox, ibox, pad_rel, out->nodes,
                                               out->d_root);
    SBR_TRY_CUDA(cudaGetLastError());
    // the cut: subtrees of at most lim primitives (about 650 of them at any n);
    // lim is at least the leaf size, so every collapsed leaf is an item of the cut
    const int64_t lim = std::max<int64_t>(std::max(leaf_max, 8), n / 400);
    if (top_sah && n > lim) {
        static std::atomic<unsigned long long> attr{0};
        SBR_TRY(set_smem_once((const void*)k_top_sah, kTopSmem, &attr));
        TopElem* E;
        int32_t* slots;
        int* cnt;
        SBR_TRY(dalloc_n(&E, kTopCap, s));
        SBR_TRY(dalloc_n(&slots, kTopCap, s));
        SBR_TRY(dalloc_n(&cnt, 2, s));
        SBR_TRY_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), s));
        ::sbr::note_launch(), k_top_cut<<<blocks_for(nn), kThreads, 0, s>>>(nn, span, hd, out->nodes, (int)lim, E, cnt,
                                                                          slots, cnt + 1);
        ::sbr::note_launch(), k_top_sah<<<1, 32 * kTopWarps, kTopSmem, s>>>(out->nodes, E, slots, cnt, cnt + 1, d_depth);
        SBR_TRY_CUDA(cudaGetLastError());
        dfree(E, s); dfree(slots, s); dfree(cnt, s);
    }
    out->order = reinterpret_cast<int32_t*>(idx);
    out->n_nodes = (int32_t)nn;
    dfree(bnd, s); dfree(part, s); dfree(hd, s); dfree(code, s); dfree(left, s); dfree(right, s); dfree(pint, s);
    dfree(pleaf, s); dfree(flag, s); dfree(span, s); dfree(lbox, s); dfree(ibox, s);
    return SBR_OK;
}

void free_lbvh(BvhNodes* b, cudaStream_t s) {
    if (b->nodes) dfree(b->nodes, s);
    if (b->order) dfree(b->order, s);
    if (b->d_root) dfree(b->d_root, s);
    *b = BvhNodes{};
}

// triangles per leaf at most: kTriLeaf, or the SBR_BVH_LEAF environment
// variable (1..16), a tuning knob for the traversal/leaf-test balance
static int tri_leaf_size() {
    const char* e = getenv("SBR_BVH_LEAF");
    if (e) {
        int v = atoi(e);
        if (v >= 1 && v <= 16) return v;
    }
    return kTriLeaf;
}

sbr_status bvh_build(const float* tri, const int32_t* surf, int64_t T, int32_t S, sbr_bvh* b, cudaStream_t s,
                     bool sah_top) {
    b->T = T;
    b->S = S;
    SBR_TRY(dalloc_n(&b->d_depth, 1, s));
    SBR_TRY(dalloc_n(&b->s_off, (size_t)S + 1, s));
    if (T == 0) {
        SBR_TRY_CUDA(cudaMemsetAsync(b->d_depth, 0, sizeof(int32_t), s));
        SBR_TRY_CUDA(cudaMemsetAsync(b->s_off, 0, sizeof(int32_t) * ((size_t)S + 1), s));
        return SBR_OK;
    }
    SBR_TRY(dalloc_n(&b->tri, 9 * T, s));
    SBR_TRY(dalloc_n(&b->surf, T, s));
    SBR_TRY(dalloc_n(&b->nrm, 3 * T, s));
    SBR_TRY(dalloc_n(&b->tri_rot, 9 * T, s));
    b->tri_sorted = b->tri_rot + 6 * T;
    SBR_TRY(dalloc_n(&b->plane_sorted, 2 * T, s));
    SBR_TRY(dalloc_n(&b->s_tri, T, s));
    float* box;
    uint32_t *key, *val;
    SBR_TRY(dalloc_n(&box, 6 * T, s));
    SBR_TRY(dalloc_n(&key, T, s));
    val = reinterpret_cast<uint32_t*>(b->s_tri);
    HostFlag* hf;
    SBR_TRY(host_flag(&hf));
    *(volatile unsigned*)hf->h = 0u;
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_tri_prep, dim3(blocks_for(T)), dim3(kThreads), 0, s, tri, surf, T, S, b->tri, b->surf, box, b->nrm,
                                                                      key, val, hf->d);
    SBR_TRY_CUDA(cudaGetLastError());
    SBR_TRY_CUDA(cudaEventRecord(hf->ev, s));
    // relative box padding: 2^-20 of (|x| + 1) covers FP32 ray/box rounding
    SBR_TRY(build_lbvh(box, T, 1.0f / (1 << 20), tri_leaf_size(), &b->tree, b->d_depth, s, sah_top));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_tri_pack, dim3(blocks_for(T)), dim3(kThreads), 0, s, b->tri, b->surf, b->nrm, b->tree.order, T,
                                                  b->tri_rot, b->plane_sorted);
    // faces per surface, ascending face id (stable sort on the surface id)
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)S) ++bits;
    SBR_TRY(radix_sort_pairs(key, val, T, bits, s));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_surface_offsets, dim3(blocks_for((int64_t)S + 1)), dim3(kThreads), 0, s, key, T, S, b->s_off);
    SBR_TRY_CUDA(cudaGetLastError());
    SBR_TRY_CUDA(cudaEventSynchronize(hf->ev));
    const unsigned h_status = *(volatile unsigned*)hf->h;
    dfree(box, s);
    dfree(key, s);
    if (h_status) {
        set_error("sbr_build_bvh: degenerate triangle or surface id out of range");
        return SBR_ERR_INVALID_ARG;
    }
    return SBR_OK;
}

}  // namespace sbr
