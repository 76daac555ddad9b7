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
#include <cstring>
#include <vector>

#include "refine.cuh"
#include "sbr_internal.cuh"

namespace sbr {
namespace {

constexpr int kThreads = 256;
inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

__global__ void k_collect(const uint32_t* __restrict__ state, size_t cap, uint32_t* __restrict__ idx,
                          unsigned int* __restrict__ count) {
    ::sbr::pdl_wait();
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

// one 32-bit sort word of slot idx[perm[i]]: the key words w[0..nf) placed at
// bit shifts sh[0..nf), surface ids shifted by one so that the -1 padding sorts
// first (the fields of one word are consecutive in significance)
struct PackWord {
    int nf;
    int w[kKeyWords];
    int sh[kKeyWords];
};
__global__ void k_key_pack(const uint32_t* __restrict__ key, const uint32_t* __restrict__ idx,
                           const uint32_t* __restrict__ perm, int64_t n, const __grid_constant__ PackWord pw,
                           uint32_t* __restrict__ out) {
    ::sbr::pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t* k = key + (size_t)idx[perm[i]] * kKeyWords;
    uint32_t v = 0;
    for (int f = 0; f < pw.nf; ++f) {
        uint32_t x = k[pw.w[f]];
        v |= (pw.w[f] >= 2 ? x + 1u : x) << pw.sh[f];
    }
    out[i] = v;
}

__global__ void k_iota(uint32_t* p, int64_t n) {
    ::sbr::pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (uint32_t)i;
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
    const float4* nodes;   // scene BVH and its BVH-order faces (containment queries)
    const float4* tris;
    double tx[3];
    const double* rx;
    const int32_t* seqf;   // [K][R] faces hit by each traced ray (refinement hints), or null
    int64_t R;             // rays of the trace (stride of seqf)
    int64_t ray0;          // first ray id of the trace
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

// one warp per key (see refine_key); lane 0 writes the validity and receiver
__global__ void k_refine(const __grid_constant__ RefineArgs a) {
    ::sbr::pdl_wait();
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
    const RefineScene sc{a.tri, a.nrm, a.s_off, a.s_tri, a.S, a.nodes, a.tris};
    const RefineOut o{a.nb_o, a.surf_o, a.face_o, a.pts_o, a.L_o, a.aod_o, a.aoa_o, a.ray_o, a.dist_o, a.jones_o};
    bool ok = refine_key<false>(lane, m, seq, v, sc, mk3(a.tx[0], a.tx[1], a.tx[2]), ld3(a.rx + 3 * rx_id), o, i);
    if (lane != 0) return;
    a.valid[i] = ok ? 1u : 0u;
    if (ok) a.rx_o[i] = rx_id;
}

// one thread per key, with the faces the kept ray hit as hints (the trace's
// per-bounce face record): the same results as k_refine
__global__ void k_refine_solo(const __grid_constant__ RefineArgs a) {
    ::sbr::pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool have = i < a.n;   // keyless lanes still take part in the warp's scans
    int rx_id = 0, m = -1;
    unsigned long long v = 0;
    int32_t seq[kKmax];
    for (int k = 0; k < kKmax; ++k) seq[k] = -1;
    if (have) {
        uint32_t slot = a.idx[a.perm[i]];
        const uint32_t* key = a.key + (size_t)slot * kKeyWords;
        v = a.val[slot];
        rx_id = (int)key[0];
        m = (int)key[1];
        for (int k = 0; k < kKmax; ++k) seq[k] = (int32_t)key[2 + k];
    }
    const RefineScene sc{a.tri, a.nrm, a.s_off, a.s_tri, a.S, a.nodes, a.tris};
    const RefineOut o{a.nb_o, a.surf_o, a.face_o, a.pts_o, a.L_o, a.aod_o, a.aoa_o, a.ray_o, a.dist_o, a.jones_o};
    const int32_t* hint = a.seqf + ((int64_t)(uint32_t)(v & 0xffffffffull) - a.ray0);
    const d3 Rx = have ? ld3(a.rx + 3 * rx_id) : mk3(0, 0, 0);
    bool ok = refine_key<true>(lane, m, seq, v, sc, mk3(a.tx[0], a.tx[1], a.tx[2]), Rx, o, have ? i : 0, hint, a.R);
    if (!have) return;
    a.valid[i] = ok ? 1u : 0u;
    if (ok) a.rx_o[i] = rx_id;
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
    ::sbr::pdl_wait();
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

// first path of each receiver (and P at n_rx), on the device and in the
// host-mapped buffer; thread 0 also stores P there
__global__ void k_rx_offsets(const int32_t* __restrict__ rx, const unsigned* __restrict__ P, int32_t n_rx,
                             int32_t* __restrict__ off, unsigned* h_P, int32_t* h_off) {
    ::sbr::pdl_wait();
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n_rx) return;
    int64_t lo = 0, hi = *P;
    if (r == 0) *(volatile unsigned*)h_P = (unsigned)hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (rx[mid] < r) lo = mid + 1; else hi = mid;
    }
    off[r] = (int32_t)lo;
    *(volatile int32_t*)(h_off + r) = (int32_t)lo;
}

// Layout of the host-mapped words of one path-list build: the key count (later
// P), the trace's alpha and final counters, then the receiver offsets.
struct MappedHead {
    unsigned count;
    unsigned pad;
    double alpha;
    TraceCountersDev cnt;
};
static_assert(sizeof(MappedHead) % 8 == 0 && sizeof(TraceCountersDev) % 8 == 0, "64-bit words");

// the key count, alpha and the trace's counters, stored to the host-mapped head
__global__ void k_peek_counts(const unsigned* __restrict__ count, const double* __restrict__ alpha,
                              const TraceCountersDev* __restrict__ cnt, MappedHead* h) {
    ::sbr::pdl_wait();
    const int i = threadIdx.x;
    constexpr int kWords = (int)(sizeof(TraceCountersDev) / 8);
    if (i < kWords)
        reinterpret_cast<volatile unsigned long long*>(&h->cnt)[i] =
            reinterpret_cast<const unsigned long long*>(cnt)[i];
    if (i == 0) {
        *(volatile unsigned*)&h->count = *count;
        *(volatile double*)&h->alpha = *alpha;
    }
}

// A pinned, device-mapped host buffer per thread and device. The small
// results the host waits for (key count, trace status, path count, receiver
// offsets) are stored there by kernels and read after the stream
// synchronisation, without copy-engine round trips.
struct Mapped {
    char* h = nullptr;
    char* d = nullptr;
    size_t cap = 0;
};

sbr_status mapped_buf(size_t bytes, char** h, char** d) {
    constexpr int kMaxDev = 64;
    thread_local Mapped m[kMaxDev];
    int dev = 0;
    SBR_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) {
        set_error("device index %d out of range", dev);
        return SBR_ERR_UNSUPPORTED;
    }
    Mapped& x = m[dev];
    if (x.cap < bytes) {
        if (x.h) {
            // every user waits for its kernels before returning; the device
            // wait also covers one that returned early on an error
            SBR_TRY_CUDA(cudaDeviceSynchronize());
            SBR_TRY_CUDA(cudaFreeHost(x.h));
            x = Mapped{};
        }
        const size_t cap = std::max<size_t>(bytes, 4096);
        SBR_TRY_CUDA(cudaHostAlloc((void**)&x.h, cap, cudaHostAllocMapped));
        SBR_TRY_CUDA(cudaHostGetDevicePointer((void**)&x.d, x.h, 0));
        x.cap = cap;
    }
    *h = x.h;
    *d = x.d;
    return SBR_OK;
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
    char *hm, *dm;
    SBR_TRY(mapped_buf(sizeof(MappedHead) + sizeof(int32_t) * (1 + (size_t)tr->n_rx), &hm, &dm));
    MappedHead* hh = reinterpret_cast<MappedHead*>(hm);
    volatile unsigned* h_count = &hh->count;
    int32_t* h_off = reinterpret_cast<int32_t*>(hm + sizeof(MappedHead));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_collect, dim3((unsigned)((cap + 255) / 256)), dim3(256), 0, s, tr->ht_state, cap, idx, count);
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_peek_counts, dim3(1), dim3(32), 0, s, count, tr->d_alpha, tr->cnt,
                                                          reinterpret_cast<MappedHead*>(dm));
    SBR_TRY_CUDA(cudaGetLastError());
    SBR_TRY_CUDA(cudaStreamSynchronize(s));
    // the trace has ended: its counters are final and are kept on the host
    memcpy(&tr->h_cnt, &hh->cnt, sizeof(TraceCountersDev));
    tr->h_alpha = hh->alpha;
    tr->h_valid = true;
    const unsigned h_trace = tr->h_cnt.status;
    // a trace that ended with an error (full dedup table, stack overflow, ...)
    // yields no path list; the table was read only as plain memory
    if (const sbr_status ts = status_from_bits(h_trace); ts != SBR_OK) {
        dfree(count, s);
        dfree(idx, s);
        return ts;
    }
    const int64_t n = *h_count;
    pl->n_keys = n;
    // sort keys: least significant word first (stable LSD over words)
    uint32_t *perm, *word;
    SBR_TRY(dalloc_n(&perm, std::max<int64_t>(n, 1), s));
    SBR_TRY(dalloc_n(&word, std::max<int64_t>(n, 1), s));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_iota, dim3(nblk(n)), dim3(kThreads), 0, s, perm, n);
    // key fields from the least significant (the last surface) to the most
    // (the receiver), packed greedily into 32-bit sort words; a stable LSD pass
    // per word, least significant word first, gives the lexicographic order
    std::vector<std::pair<int, int>> fields;  // (key word, bits)
    for (int k = K - 1; k >= 0; --k) fields.push_back({2 + k, bits_for((int64_t)b->S)});
    fields.push_back({1, bits_for(K)});
    fields.push_back({0, bits_for(std::max(1, tr->n_rx - 1))});
    size_t f0 = 0;
    while (f0 < fields.size()) {
        PackWord pw{};
        int bits = 0;
        while (f0 < fields.size() && bits + fields[f0].second <= 32) {
            pw.w[pw.nf] = fields[f0].first;
            pw.sh[pw.nf] = bits;
            bits += fields[f0].second;
            ++pw.nf;
            ++f0;
        }
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_key_pack, dim3(nblk(n)), dim3(kThreads), 0, s, tr->ht_key, idx, perm, n, pw, word);
        SBR_TRY_CUDA(cudaGetLastError());
        SBR_TRY(radix_sort_pairs(word, perm, n, bits, s));
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
    a.nodes = b->T > 0 ? b->tree.nodes : nullptr;
    a.tris = b->tri_sorted;
    for (int k = 0; k < 3; ++k) a.tx[k] = tr->params.tx[k];
    a.rx = tr->rx;
    a.seqf = tr->seqf;
    a.R = tr->Rr;
    a.ray0 = tr->ray0;
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
        if (a.seqf)
            // one warp per block: the keys spread over every SM (latency-bound FP64 chains)
            ::sbr::note_launch(), (void)::sbr::launch_pdl(k_refine_solo, dim3((unsigned)((n + 31) / 32)), dim3(32), 0, s, a);
        else
            ::sbr::note_launch(), (void)::sbr::launch_pdl(k_refine, dim3(nblk(32 * n)), dim3(kThreads), 0, s, a);
        SBR_TRY_CUDA(cudaGetLastError());
        SBR_TRY_CUDA(cudaMemcpyAsync(pos, valid, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    SBR_TRY(exclusive_scan_u32(pos, n, count, s));
    // the list is sized for every key (P <= n), so compaction and the receiver
    // offsets run before the host learns P: one wait for P and the offsets
    const int64_t Pp = nn;
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
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_compact_all, dim3(nblk(32 * n)), dim3(kThreads), 0, s, c);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_rx_offsets, dim3(nblk((int64_t)tr->n_rx + 1)), dim3(kThreads), 0, s,
        pl->rx, count, tr->n_rx, pl->rx_off, &reinterpret_cast<MappedHead*>(dm)->count,
        reinterpret_cast<int32_t*>(dm + sizeof(MappedHead)));
    SBR_TRY_CUDA(cudaGetLastError());
    pl->h_rx_off = new int32_t[tr->n_rx + 1];
    SBR_TRY_CUDA(cudaStreamSynchronize(s));
    memcpy(pl->h_rx_off, h_off, sizeof(int32_t) * (tr->n_rx + 1));
    const int64_t P = *h_count;
    pl->P = P;
    pl->n_invalid = n - P;
    dfree(count, s); dfree(idx, s); dfree(perm, s); dfree(word, s); dfree(valid, s); dfree(pos, s);
    dfree(a.rx_o, s); dfree(a.nb_o, s); dfree(a.surf_o, s); dfree(a.face_o, s); dfree(a.pts_o, s);
    dfree(a.L_o, s); dfree(a.aod_o, s); dfree(a.aoa_o, s); dfree(a.ray_o, s); dfree(a.dist_o, s);
    dfree(a.jones_o, s);
    return SBR_OK;
}

}  // namespace sbr
