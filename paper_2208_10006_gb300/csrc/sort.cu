// Device sort and scan primitives used by the BVH build (Morton order,
// surface CSR) and by path compaction (key order, valid-path compaction).
//
// radix_sort_pairs: stable LSD radix sort, 8-bit digits. Each pass: digit
// counts per tile, their exclusive scan (digit-major), and a stable scatter.
// Up to 12,288 keys the whole sort runs in one block in shared memory; above
// that in one cooperative launch (two grid-wide barriers per pass, every
// block forming its own offsets from all tiles' counts); where a cooperative
// launch is not available, as separate launches per phase.
#include <algorithm>
#include <atomic>
#include <cstdlib>

#include <cooperative_groups.h>

#include "sbr_internal.cuh"

namespace cg = cooperative_groups;

namespace sbr {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 elements per block
constexpr int kScanBlock = 1024;

// digit counts of tile t (kSortTile keys from t * kSortTile), digit-major:
// hist[d * ntiles + t]
__device__ __forceinline__ void tile_hist(const uint32_t* keys, int64_t n, int shift, uint32_t* hist, int ntiles,
                                          int t) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)t * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + t] = h[threadIdx.x];
    __syncthreads();
}

// stable scatter of tile t, its digits starting at the scanned hist[d * ntiles + t]
__device__ __forceinline__ void tile_scatter(const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                                             uint32_t* vout, int64_t n, int shift, const uint32_t* hist,
                                             int ntiles, int t) {
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_warp[kSortThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_run[tid] = hist[(int64_t)tid * ntiles + t];
    int64_t base = (int64_t)t * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
        for (int w = 0; w < kSortThreads / 32; ++w) s_warp[w][tid] = 0;
        __syncthreads();
        int64_t i = base + r * kSortThreads + tid;
        bool valid = i < n;
        uint32_t k = valid ? kin[i] : 0u, v = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) s_warp[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = s_run[tid];
            for (int w = 0; w < kSortThreads / 32; ++w) {
                uint32_t c = s_warp[w][tid];
                s_warp[w][tid] = run;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_warp[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
}

__global__ void k_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                       uint32_t* __restrict__ hist, int nblocks) {
    ::sbr::pdl_wait();
    tile_hist(keys, n, shift, hist, nblocks, blockIdx.x);
}

__global__ void k_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                          uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                          int shift, const uint32_t* __restrict__ hist, int nblocks) {
    ::sbr::pdl_wait();
    tile_scatter(kin, vin, kout, vout, n, shift, hist, nblocks, blockIdx.x);
}

// block-level exclusive scan of up to kScanBlock values
__device__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* total) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? warp_sums[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < nw) warp_sums[lane] = si - s;
        if (lane == nw - 1) s_total = si;
    }
    __syncthreads();
    uint32_t res = warp_sums[warp] + incl - x;
    if (total) *total = s_total;
    __syncthreads();
    return res;
}

__global__ void k_scan_blocks(uint32_t* data, int64_t n, uint32_t* block_sums) {
    ::sbr::pdl_wait();
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    uint32_t x = i < n ? data[i] : 0u;
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(x, &tot);
    if (i < n) data[i] = ex;
    if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = tot;
}

__global__ void k_add_offsets(uint32_t* data, int64_t n, const uint32_t* offs) {
    ::sbr::pdl_wait();
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) data[i] += offs[blockIdx.x];
}

__global__ void k_total(const uint32_t* scanned, const uint32_t* last_in, int64_t n,
                        uint32_t* total) {
    ::sbr::pdl_wait();
    *total = n > 0 ? scanned[n - 1] + *last_in : 0u;
}

// The sort of a mid-sized array in one cooperative launch (every block is
// resident), one tile of 256 x rounds keys per block and one chunk of
// 32 x rounds keys per warp. Per 8-bit pass: each warp counts the digits of
// its chunk into shared memory and the block publishes its tile's counts
// (tile-major); after a grid-wide barrier every block forms its own offsets,
// digit base (exclusive scan over digits of the counts of all tiles) + the
// counts of the tiles before it + those of its warps before each warp; then
// every warp scatters its chunk in rounds of 32, equal digits ranked by lane,
// which keeps the pass stable; a second barrier ends the pass. Data written
// by other blocks is read at L2 (__ldcg). The result ends in (k0, v0).
constexpr int kCoopTileMin = 1024;   // keys per tile at least (fewer, larger tiles: fewer counts to add)
constexpr int kCoopMaxRounds = 32;   // rounds of 32 keys per warp at most

__global__ void __launch_bounds__(kSortThreads)
k_sort_coop(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n, int passes, int rounds,
            uint32_t* hist) {
    cg::grid_group grid = cg::this_grid();
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t s_cnt[kWarps][256];   // per warp and digit: count, then output position
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int ntiles = (int)gridDim.x, t = (int)blockIdx.x;
    const int64_t chunk = 32 * (int64_t)rounds;
    const int64_t c0 = min(n, ((int64_t)t * kWarps + warp) * chunk), c1 = min(n, c0 + chunk);
    uint32_t *ka = k0, *va = v0, *kb = k1, *vb = v1;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        for (int d = lane; d < 256; d += 32) s_cnt[warp][d] = 0;
        __syncwarp();
        for (int64_t b = c0; b < c1; b += 32) {
            const int64_t i = b + lane;
            const uint32_t d = i < c1 ? ((__ldcg(ka + i) >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && (peers & lt) == 0) s_cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            uint32_t c = 0;
            for (int w = 0; w < kWarps; ++w) c += s_cnt[w][tid];
            hist[(int64_t)t * 256 + tid] = c;
        }
        grid.sync();
        {
            // digit tid: its count over all tiles and over the tiles before t
            uint32_t total = 0, before = 0;
            int u = 0;
            for (; u + 4 <= ntiles; u += 4) {
                const uint32_t x0 = __ldcg(hist + (int64_t)u * 256 + tid);
                const uint32_t x1 = __ldcg(hist + (int64_t)(u + 1) * 256 + tid);
                const uint32_t x2 = __ldcg(hist + (int64_t)(u + 2) * 256 + tid);
                const uint32_t x3 = __ldcg(hist + (int64_t)(u + 3) * 256 + tid);
                total += x0 + x1 + x2 + x3;
                before += (u < t ? x0 : 0u) + (u + 1 < t ? x1 : 0u) + (u + 2 < t ? x2 : 0u) + (u + 3 < t ? x3 : 0u);
            }
            for (; u < ntiles; ++u) {
                const uint32_t x = __ldcg(hist + (int64_t)u * 256 + tid);
                total += x;
                before += u < t ? x : 0u;
            }
            uint32_t run = block_exclusive_scan(total, nullptr) + before;
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = s_cnt[w][tid];
                s_cnt[w][tid] = run;
                run += c;
            }
        }
        __syncthreads();
        for (int64_t b = c0; b < c1; b += 32) {
            const int64_t i = b + lane;
            const bool valid = i < c1;
            const uint32_t k = valid ? __ldcg(ka + i) : 0u, v = valid ? __ldcg(va + i) : 0u;
            const uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid) {
                const uint32_t pos = s_cnt[warp][d] + __popc(peers & lt);
                kb[pos] = k;
                vb[pos] = v;
            }
            __syncwarp();
            if (valid && (peers & lt) == 0) s_cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        grid.sync();
        uint32_t* q = ka; ka = kb; kb = q;
        q = va; va = vb; vb = q;
    }
    if (ka != k0)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            k0[i] = __ldcg(ka + i);
            v0[i] = __ldcg(va + i);
        }
}

sbr_status scan_rec(uint32_t* data, int64_t n, cudaStream_t s) {
    if (n <= 0) return SBR_OK;
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 1) {
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_scan_blocks, dim3(1), dim3(kScanBlock), 0, s, data, n, nullptr);
        SBR_TRY_CUDA(cudaGetLastError());
        return SBR_OK;
    }
    uint32_t* sums;
    SBR_TRY(dalloc_n(&sums, nb, s));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_scan_blocks, dim3((unsigned)nb), dim3(kScanBlock), 0, s, data, n, sums);
    SBR_TRY_CUDA(cudaGetLastError());
    sbr_status st = scan_rec(sums, nb, s);
    if (st == SBR_OK) {
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_add_offsets, dim3((unsigned)nb), dim3(kScanBlock), 0, s, data, n, sums);
        if (cudaGetLastError() != cudaSuccess) st = SBR_ERR_CUDA;
    }
    dfree(sums, s);
    return st;
}

// Whole sort of a small array in one block: keys and values live in shared
// memory and every 8-bit pass runs in the same launch. Warp w owns the
// contiguous chunk [w c, (w+1) c) of the array, so a pass needs three block
// barriers: per-warp digit counts, their scan (digit-major over warps, then
// over digits), and the stable scatter, where each warp walks its chunk in
// rounds of 32 and ranks equal digits of a round by lane.
constexpr int kSmallThreads = 1024;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallMax = 12288;  // 2 x 2 x 4 B x 12288 = 192 KB of shared memory

__global__ void __launch_bounds__(kSmallThreads)
k_sort_small(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int n, int passes) {
    ::sbr::pdl_wait();
    extern __shared__ uint32_t sm[];
    uint32_t* ka = sm;
    uint32_t* va = sm + kSmallMax;
    uint32_t* kb = sm + 2 * kSmallMax;
    uint32_t* vb = sm + 3 * kSmallMax;
    __shared__ uint32_t s_cnt[kSmallWarps][256];   // per warp and digit: count, then output position
    __shared__ uint32_t s_wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int chunk = ((n + kSmallWarps - 1) / kSmallWarps + 31) & ~31;
    const int c0 = min(n, warp * chunk), c1 = min(n, c0 + chunk);
    for (int i = tid; i < n; i += kSmallThreads) { ka[i] = keys[i]; va[i] = vals[i]; }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        for (int d = lane; d < 256; d += 32) s_cnt[warp][d] = 0;
        __syncwarp();
        for (int base = c0; base < c1; base += 32) {
            const int i = base + lane;
            const uint32_t d = i < c1 ? ((ka[i] >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && (peers & lt) == 0) s_cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t run = 0, incl = 0;
        if (tid < 256) {
            for (int w = 0; w < kSmallWarps; ++w) {
                const uint32_t c = s_cnt[w][tid];
                s_cnt[w][tid] = run;
                run += c;
            }
            incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[warp] = incl;
        }
        __syncthreads();
        if (tid < 256) {
            uint32_t off = incl - run;
            for (int k = 0; k < warp; ++k) off += s_wsum[k];
            for (int w = 0; w < kSmallWarps; ++w) s_cnt[w][tid] += off;
        }
        __syncthreads();
        for (int base = c0; base < c1; base += 32) {
            const int i = base + lane;
            const bool valid = i < c1;
            const uint32_t k = valid ? ka[i] : 0u, v = valid ? va[i] : 0u;
            const uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid) {
                const uint32_t pos = s_cnt[warp][d] + __popc(peers & lt);
                kb[pos] = k;
                vb[pos] = v;
            }
            __syncwarp();
            if (valid && (peers & lt) == 0) s_cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t* t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    for (int i = tid; i < n; i += kSmallThreads) { keys[i] = ka[i]; vals[i] = va[i]; }
}

}  // namespace

sbr_status exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* total, cudaStream_t s) {
    if (n <= 0) {
        if (total) SBR_TRY_CUDA(cudaMemsetAsync(total, 0, sizeof(uint32_t), s));
        return SBR_OK;
    }
    uint32_t* last = nullptr;
    if (total) {
        SBR_TRY(dalloc_n(&last, 1, s));
        SBR_TRY_CUDA(cudaMemcpyAsync(last, data + n - 1, sizeof(uint32_t),
                                     cudaMemcpyDeviceToDevice, s));
    }
    sbr_status st = scan_rec(data, n, s);
    if (st == SBR_OK && total) {
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_total, dim3(1), dim3(1), 0, s, data, last, n, total);
        if (cudaGetLastError() != cudaSuccess) st = SBR_ERR_CUDA;
    }
    if (last) dfree(last, s);
    return st;
}

// blocks of k_sort_coop that fit on the current device at once (0: no
// cooperative launch there)
static sbr_status coop_blocks(int* out) {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];   // blocks + 1; 0 = not yet known
    int dev = 0;
    SBR_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) { *out = 0; return SBR_OK; }
    int c = cache[dev].load();
    if (c == 0) {
        int coop = 0, sms = 0, per_sm = 0;
        SBR_TRY_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        SBR_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        SBR_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_coop, kSortThreads, 0));
        c = (coop ? sms * per_sm : 0) + 1;
        cache[dev].store(c);
    }
    *out = c - 1;
    return SBR_OK;
}

sbr_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return SBR_OK;
    if (n > 0x7fffffffLL) {
        set_error("radix_sort_pairs: n too large");
        return SBR_ERR_UNSUPPORTED;
    }
    if (n <= kSmallMax) {
        const size_t smem = sizeof(uint32_t) * 4 * kSmallMax;
        static std::atomic<unsigned long long> attr{0};
        SBR_TRY(set_smem_once((const void*)k_sort_small, (int)smem, &attr));
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_sort_small, dim3(1), dim3(kSmallThreads), smem, s, keys, vals, (int)n, (bits + 7) / 8);
        SBR_TRY_CUDA(cudaGetLastError());
        return SBR_OK;
    }
    int passes = (bits + 7) / 8;
    int coop = 0;
    // SBR_SORT_PHASES=1 (read at each call) keeps to the per-phase launches: a
    // test hook for the path taken where no cooperative launch is available
    const char* force = getenv("SBR_SORT_PHASES");
    if (!(force && force[0] == '1')) SBR_TRY(coop_blocks(&coop));
    // cooperative: one tile of 256 x rounds keys per block, every block resident
    const int64_t coop_tiles = std::min<int64_t>(coop, (n + kCoopTileMin - 1) / kCoopTileMin);
    const int64_t rounds = coop_tiles > 0 ? (n + 256 * coop_tiles - 1) / (256 * coop_tiles) : 0;
    if (coop_tiles > 0 && rounds <= kCoopMaxRounds) {
        int grid = (int)coop_tiles, r = (int)rounds;
        uint32_t *k2, *v2, *hist;
        SBR_TRY(dalloc_n(&k2, n, s));
        SBR_TRY(dalloc_n(&v2, n, s));
        SBR_TRY(dalloc_n(&hist, (size_t)256 * grid, s));
        void* args[] = {&keys, &vals, &k2, &v2, &n, &passes, &r, &hist};
        ::sbr::note_launch();
        SBR_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)k_sort_coop, dim3(grid), dim3(kSortThreads), args, 0, s));
        dfree(k2, s);
        dfree(v2, s);
        dfree(hist, s);
        return SBR_OK;
    }
    int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    uint32_t *k2, *v2, *hist;
    SBR_TRY(dalloc_n(&k2, n, s));
    SBR_TRY(dalloc_n(&v2, n, s));
    SBR_TRY(dalloc_n(&hist, (size_t)256 * nblocks, s));
    uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
    sbr_status st = SBR_OK;
    for (int p = 0; p < passes && st == SBR_OK; ++p) {
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_hist, dim3(nblocks), dim3(kSortThreads), 0, s, ka, n, 8 * p, hist, nblocks);
        st = scan_rec(hist, (int64_t)256 * nblocks, s);
        if (st != SBR_OK) break;
        ::sbr::note_launch(), (void)::sbr::launch_pdl(k_scatter, dim3(nblocks), dim3(kSortThreads), 0, s, ka, va, kb, vb, n, 8 * p, hist, nblocks);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("radix scatter launch failed");
            st = SBR_ERR_CUDA;
        }
        uint32_t* t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (st == SBR_OK && ka != keys) {
        cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
    dfree(k2, s);
    dfree(v2, s);
    dfree(hist, s);
    return st;
}

}  // namespace sbr
