// Batched execution of many Tx-Rx jobs over several scenes (the C ABI's
// sbr_batch_*): the per-job pipeline of sbr_trace, sbr_paths, sbr_path_gains
// and sbr_synthesize_H (Sec. II-A, Eq. 1, 3, 6-10, 13-14) run for all jobs of
// a wave at once.
//
// Jobs are grouped, in order, into waves whose rays fit the ray-queue
// capacity. Per wave:
//   1. K_max + 1 persistent bounce launches over every ray of every job of
//      the wave (trace.cu, k_trace_batch), one shared dedup table whose key
//      carries the job index;
//   2. k_batch_collect: the table's keys go to per-job slot lists;
//   3. k_batch_paths: one CTA per job sorts its keys in shared memory, refines
//      them (one warp per key, the refinement of sbr_paths), and compacts the
//      valid ones into the job's path store;
//   4. k_batch_gains: (job, 32-frequency) tiles compute the gains and the
//      synthesis weights w = g exp(-j 2 pi frac(f L / c));
//   5. k_batch_delays: per job, the FP32 element delays of the synthesis;
//   6. the tensor-core synthesis over the (job, frequency, tile) items of the
//      wave (synth_tc.cu);
//   7. k_batch_status: the wave's device status bits go to its jobs.
// Every buffer is allocated by sbr_batch_create and every size a kernel needs
// is read on the device, so the whole batch is captured once into a CUDA graph
// and replayed by one graph launch per run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "batch.cuh"
#include "synth_ops.cuh"
#include "dfloat.cuh"
#include "gains.cuh"
#include "refine.cuh"

struct sbr_batch;

namespace sbr {
namespace {

constexpr int kBThreads = 256;
constexpr int kGainTileF = 32;   // frequencies per gain tile
constexpr int kKeySortWords = kKeyWords - 1;   // n_bounce and the surface sequence

// ---------------------------------------------------------------- kernels
__global__ void k_batch_collect(const uint32_t* __restrict__ state, const uint32_t* __restrict__ key,
                                size_t cap, int32_t* __restrict__ nkeys, uint32_t* __restrict__ slots,
                                int32_t path_cap, unsigned int* __restrict__ status) {
    size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= cap || state[s] != 2u) return;
    int job = (int)key[s * kKeyWords];
    int pos = atomicAdd(&nkeys[job], 1);
    if (pos < path_cap) slots[(int64_t)job * path_cap + pos] = (uint32_t)s;
    else atomicOr(&status[job], (unsigned)ST_CAPACITY);
}

// exclusive scan of flag[0..m) into pos[0..m) by the whole CTA; returns the total
__device__ int cta_exclusive_scan(const int32_t* flag, int32_t* pos, int m, int* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int base = 0;
    for (int c0 = 0; c0 < m; c0 += kBThreads) {
        int r = c0 + tid;
        int v = r < m ? flag[r] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int t = lane < kBThreads / 32 ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < kBThreads / 32) wsum[lane] = t;
        }
        __syncthreads();
        int wb = warp > 0 ? wsum[warp - 1] : 0;
        if (r < m) pos[r] = base + wb + x - v;
        int tot = wsum[kBThreads / 32 - 1];
        __syncthreads();
        base += tot;
    }
    return base;
}

struct BatchPathArgs {
    const BatchJobDev* jobs;     // wave's jobs
    const int32_t* nkeys;        // [wave jobs]
    const uint32_t* slots;       // [wave jobs][path_cap]
    const uint32_t* ht_key;
    const unsigned long long* ht_val;
    int32_t path_cap;
    RefineOut raw;               // wave-local records [wave job * path_cap + sorted position]
    const void* raw_f[10];       // the same fields as untyped arrays, for the compaction
    void* fin_f[10];             // batch path store
    int words[10];               // 32-bit words per record of each field
    int32_t* np;                 // [wave jobs]
};

// one CTA per job: rank sort of its keys, refinement, compaction
__global__ void __launch_bounds__(kBThreads) k_batch_paths(const __grid_constant__ BatchPathArgs a) {
    extern __shared__ uint32_t sh[];
    __shared__ int wsum[kBThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jl = blockIdx.x;
    const BatchJobDev* J = a.jobs + jl;
    const int m = min(a.nkeys[jl], a.path_cap);
    uint32_t* kw = sh;                                            // [path_cap][kKeySortWords]
    int32_t* order = (int32_t*)(kw + (size_t)kKeySortWords * a.path_cap);
    int32_t* valid = order + a.path_cap;
    int32_t* pos = valid + a.path_cap;
    const uint32_t* slots = a.slots + (int64_t)jl * a.path_cap;
    // sortable key words: n_bounce, then surfaces shifted by one (padding first),
    // the order sbr_paths sorts a receiver's keys in
    for (int i = tid; i < m; i += kBThreads) {
        const uint32_t* key = a.ht_key + (size_t)slots[i] * kKeyWords;
        for (int w = 0; w < kKeySortWords; ++w) {
            uint32_t v = key[1 + w];
            kw[i * kKeySortWords + w] = w >= 1 ? v + 1u : v;
        }
    }
    __syncthreads();
    for (int i = tid; i < m; i += kBThreads) {
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            int lt = 0;
            for (int w = 0; w < kKeySortWords; ++w) {
                uint32_t x = kw[j * kKeySortWords + w], y = kw[i * kKeySortWords + w];
                if (x != y) { lt = x < y; break; }
            }
            rank += lt;
        }
        order[rank] = i;   // keys are distinct: ranks are a permutation
    }
    __syncthreads();
    const RefineScene sc{J->tri, J->nrm, J->s_off, J->s_tri, J->S, J->nodes, J->tris};
    const d3 Tx = mk3(J->tx[0], J->tx[1], J->tx[2]);
    const d3 Rx = mk3(J->rx[0], J->rx[1], J->rx[2]);
    const int64_t rb = (int64_t)jl * a.path_cap;
    for (int r = warp; r < m; r += kBThreads / 32) {
        const uint32_t slot = slots[order[r]];
        const uint32_t* key = a.ht_key + (size_t)slot * kKeyWords;
        int32_t seq[kKmax];
        for (int k = 0; k < kKmax; ++k) seq[k] = (int32_t)key[2 + k];
        bool ok = refine_key<false>(lane, (int)key[1], seq, a.ht_val[slot], sc, Tx, Rx, a.raw, rb + r);
        if (lane == 0) valid[r] = ok ? 1 : 0;
    }
    __syncthreads();
    const int P = cta_exclusive_scan(valid, pos, m, wsum);
    for (int r = warp; r < m; r += kBThreads / 32) {
        if (!valid[r]) continue;
        const int64_t src = rb + r, dst = J->path_base + pos[r];
        for (int f = 0; f < 10; ++f) {
            const uint32_t* sp = static_cast<const uint32_t*>(a.raw_f[f]) + src * a.words[f];
            uint32_t* dp = static_cast<uint32_t*>(a.fin_f[f]) + dst * a.words[f];
            for (int w = lane; w < a.words[f]; w += 32) dp[w] = sp[w];
        }
    }
    if (tid == 0) a.np[jl] = P;
}

// row length of a job's synthesis operands (weights, transposed delays): the
// path capacity rounded up to the 8-path K-steps the tensor-core form reads
inline int32_t synth_stride(int32_t path_cap) { return (path_cap + 7) & ~7; }

struct BatchGainArgs {
    const BatchJobDev* jobs;
    const int32_t* tile_job;     // wave-local job of each tile
    const int32_t* tile_f0;      // first frequency of each tile
    const int32_t* np;           // [wave jobs]
    BatchPathsDev paths;
    float2* g;
    float2* w;
    float2* wl;
    float* sc;
    int32_t path_cap;            // row length of w: synth_stride(the path capacity)
};

// the gain of sbr_path_gains and the synthesis weights (synth_ops.cuh, the
// arithmetic of the single-receiver form), per (path, frequency) of a (job,
// 32-frequency) tile: reflected-path weights w (padded slots up to the next
// multiple of 8 zeroed), the LoS weight wl and the FP16 scale sc per frequency
__global__ void __launch_bounds__(kBThreads) k_batch_gains(const __grid_constant__ BatchGainArgs a) {
    __shared__ unsigned s_max[kGainTileF];
    const int jl = a.tile_job[blockIdx.x], f0 = a.tile_f0[blockIdx.x];
    const BatchJobDev* J = a.jobs + jl;
    const int P = a.np[jl], F = J->F;
    const int nf = min(kGainTileF, F - f0);
    const int n0 = (P > 0 && a.paths.nb[J->path_base] == 0) ? 1 : 0;   // the LoS path sorts first
    const int nrefl = P - n0, npad = (nrefl + 7) & ~7;
    if (threadIdx.x < kGainTileF) s_max[threadIdx.x] = 0u;
    __syncthreads();
    for (int it = threadIdx.x; it < P * nf; it += kBThreads) {
        const int p = it / nf, f = f0 + (it - p * nf);
        const int64_t slot = J->path_base + p;
        const double fr = J->freqs[f];
        const double L = a.paths.L[slot];
        float2 gg = path_gain(a.paths.nb[slot], a.paths.surf + slot * kKmax, L, a.paths.jones + slot * kJones,
                              J->mats, J->S, fr, J->gamma ? J->gamma + f : nullptr,
                              J->disp ? J->disp + f : nullptr, J->pol);
        a.g[J->g_base + (int64_t)p * F + f] = gg;
        const float2 ww = synth_weight(gg, fr, L);
        if (p < n0) {
            a.wl[J->wl_base + f] = ww;
        } else {
            a.w[J->w_base + (int64_t)f * a.path_cap + (p - n0)] = ww;
            atomicMax(&s_max[f - f0], __float_as_uint(fmaxf(fabsf(ww.x), fabsf(ww.y))));
        }
    }
    for (int it = threadIdx.x; it < (npad - nrefl) * nf; it += kBThreads) {
        const int n = nrefl + it / nf, f = f0 + it % nf;
        a.w[J->w_base + (int64_t)f * a.path_cap + n] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    if ((int)threadIdx.x < nf) {
        const int f = f0 + threadIdx.x;
        a.sc[J->wl_base + f] = synth_scale(__uint_as_float(s_max[threadIdx.x]));
        if (n0 == 0) a.wl[J->wl_base + f] = make_float2(0.f, 0.f);
    }
}

// element delays of the synthesis (Eq. 13-14 near field; synth_ops.cuh), FP64
// then FP32, transposed per element over the reflected paths (padded slots up
// to the next multiple of 8 zeroed):
//   dt[p][n] = |T_p - P1| - |T_0 - P1|, dr[q][n] = |R_q - Pm| - |R_0 - Pm|;
//   dl[q][p] = |T_p - R_q| - |T_0 - R_0|
__global__ void __launch_bounds__(kBThreads) k_batch_delays(const BatchJobDev* __restrict__ jobs,
                                                            const int32_t* __restrict__ np, BatchPathsDev paths,
                                                            int32_t path_cap, float* __restrict__ dt,
                                                            float* __restrict__ dr, float* __restrict__ dl) {
    const BatchJobDev* J = jobs + blockIdx.x;
    const int P = np[blockIdx.x], Nt = J->Nt, Nr = J->Nr;
    const d3 T0 = mk3(J->tx[0], J->tx[1], J->tx[2]), R0 = mk3(J->rx[0], J->rx[1], J->rx[2]);
    const int n0 = (P > 0 && paths.nb[J->path_base] == 0) ? 1 : 0;
    const int nrefl = P - n0, npad = (nrefl + 7) & ~7;
    const int ne = Nt + Nr;
    // one thread per (path, element side, run of up to 8 elements)
    const int gt = (Nt + 7) / 8, gr = (Nr + 7) / 8;
    for (int it = threadIdx.x; it < npad * (gt + gr); it += kBThreads) {
        const int n = it % npad, g = it / npad;
        const bool tx = g < gt;
        const int e0 = (tx ? g : g - gt) * 8, e1 = min(tx ? Nt : Nr, e0 + 8);
        // element e, path n at [n / 4][e][n % 4] (layout in synth_ops.cuh)
        float* dst = (tx ? dt + J->dt_base : dr + J->dr_base) + (int64_t)(n >> 2) * (tx ? Nt : Nr) * 4 + (n & 3);
        if (n < nrefl) {
            const int64_t slot = J->path_base + n + n0;
            const int m = paths.nb[slot];
            const d3 Pk = ld3(paths.pts + (slot * kKmax + (tx ? 0 : m - 1)) * 3);
            const double ref = dist_rn(tx ? T0 : R0, Pk);
            const double* el = tx ? J->tx_elem : J->rx_elem;
            for (int e = e0; e < e1; ++e) dst[(int64_t)e * 4] = el_delay(el + 3 * e, Pk, ref);
        } else {
            for (int e = e0; e < e1; ++e) dst[(int64_t)e * 4] = 0.f;
        }
    }
    (void)ne;
    const double ref = dist_rn(T0, R0);
    for (int it = threadIdx.x; it < Nr * Nt; it += kBThreads) {
        const int q = it / Nt, p = it - q * Nt;
        dl[J->dl_base + it] = el_delay(J->tx_elem + 3 * p, ld3(J->rx_elem + 3 * q), ref);
    }
}

__global__ void k_batch_status(const TraceCountersDev* __restrict__ cnt, int32_t n_jobs,
                               unsigned int* __restrict__ status) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_jobs) status[j] |= cnt->status;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ---------------------------------------------------------------- per-N launch data
// alpha of every subdivision used by a batch, kept for the process
struct NData {
    double alpha = 0.0;
};
std::mutex g_nmu;
std::map<std::pair<int, int>, NData> g_ndata;   // (device, N)

sbr_status ndata(int N, cudaStream_t s, NData* out) {
    int dev = 0;
    SBR_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_nmu);
    auto it = g_ndata.find({dev, N});
    if (it == g_ndata.end()) {
        NData d;
        double* da = nullptr;
        sbr_status st = dalloc_n(&da, 1, s);
        if (st == SBR_OK) st = launch_alpha_fast(N, da, s);
        if (st == SBR_OK && cudaMemcpyAsync(&d.alpha, da, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = SBR_ERR_CUDA;
        if (st == SBR_OK && cudaStreamSynchronize(s) != cudaSuccess) st = SBR_ERR_CUDA;
        if (da) dfree(da, s);
        if (st != SBR_OK) {
            if (st == SBR_ERR_CUDA) set_error("alpha of N=%d failed", N);
            return st;
        }
        it = g_ndata.emplace(std::make_pair(dev, N), d).first;
    }
    *out = it->second;
    return SBR_OK;
}

struct Wave {
    int j0 = 0, j1 = 0;
    int64_t R_total = 0;
    int Kmax = 0;
    int64_t seq_words = 0;
    int64_t items = 0;
    int n_tiles = 0;
    int64_t dt_words = 0, dr_words = 0, dl_words = 0, w_words = 0;
    int64_t* d_ray_off = nullptr;
    int64_t* d_item_off = nullptr;
    int32_t* d_tile_job = nullptr;
    int32_t* d_tile_f0 = nullptr;
    TraceCountersDev* cnt = nullptr;
};

template <class T>
sbr_status dmalloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("batch allocation of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
        return SBR_ERR_ALLOC;
    }
    return SBR_OK;
}

}  // namespace
}  // namespace sbr

struct sbr_batch {
    int device = 0;
    sbr_batch_config cfg{};
    int32_t n_jobs = 0;
    std::vector<sbr_batch_job> jobs;
    std::vector<sbr::Wave> waves;
    int64_t rays = 0;
    int max_wave_jobs = 0;
    std::vector<void*> owned;           // every cudaMalloc of the batch
    sbr::BatchJobDev* d_jobs = nullptr;
    // trace
    void* q0 = nullptr;
    void* q1 = nullptr;
    int32_t* seq = nullptr;
    uint32_t* ht_state = nullptr;
    uint32_t* ht_key = nullptr;
    unsigned long long* ht_val = nullptr;
    uint32_t ht_mask = 0;
    // paths
    int32_t* nkeys = nullptr;           // [n_jobs]
    uint32_t* slots = nullptr;          // [max wave jobs * path_cap]
    sbr::BatchPathsDev raw{};           // [max wave jobs * path_cap]
    sbr::BatchPathsDev fin{};           // [n_jobs * path_cap]
    int32_t* np = nullptr;              // [n_jobs]
    unsigned int* status = nullptr;     // [n_jobs]
    float2* g = nullptr;
    std::vector<int64_t> g_base;
    // synthesis scratch
    float* dt = nullptr;
    float* dr = nullptr;
    float* dl = nullptr;
    float2* w = nullptr;
    float2* wl = nullptr;
    float* sc = nullptr;
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
};

namespace sbr {
namespace {

template <class T>
sbr_status balloc(sbr_batch* b, T** p, size_t n) {
    SBR_TRY(dmalloc(p, n));
    b->owned.push_back(*p);
    return SBR_OK;
}

sbr_status alloc_paths(sbr_batch* b, BatchPathsDev* d, size_t n) {
    SBR_TRY(balloc(b, &d->nb, n));
    SBR_TRY(balloc(b, &d->surf, n * kKmax));
    SBR_TRY(balloc(b, &d->face, n * kKmax));
    SBR_TRY(balloc(b, &d->pts, n * kKmax * 3));
    SBR_TRY(balloc(b, &d->L, n));
    SBR_TRY(balloc(b, &d->aod, n * 2));
    SBR_TRY(balloc(b, &d->aoa, n * 2));
    SBR_TRY(balloc(b, &d->ray, n));
    SBR_TRY(balloc(b, &d->dist, n));
    SBR_TRY(balloc(b, &d->jones, n * kJones));
    return SBR_OK;
}

void free_batch(sbr_batch* b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void* p : b->owned) cudaFree(p);
    cudaSetDevice(cur);
    delete b;
}

size_t path_smem(int path_cap) { return (size_t)path_cap * (kKeySortWords + 3) * sizeof(uint32_t); }

// every launch of one run, on s (capturable: no allocation, no synchronisation)
sbr_status enqueue(sbr_batch* b, cudaStream_t s) {
    const sbr_batch_config& c = b->cfg;
    const bool f16 = c.precision != SBR_SYNTH_BF16X3;
    SBR_TRY_CUDA(cudaMemsetAsync(b->status, 0, sizeof(unsigned) * b->n_jobs, s));
    SBR_TRY_CUDA(cudaMemsetAsync(b->nkeys, 0, sizeof(int32_t) * b->n_jobs, s));
    SBR_TRY_CUDA(cudaMemsetAsync(b->np, 0, sizeof(int32_t) * b->n_jobs, s));
    for (const Wave& wv : b->waves) {
        const int nj = wv.j1 - wv.j0;
        const BatchJobDev* jobs = b->d_jobs + wv.j0;
        BatchTraceWave tw{};
        tw.ico = make_ico_lattice();
        tw.jobs = jobs;
        tw.ray_off = wv.d_ray_off;
        tw.n_jobs = nj;
        tw.Kmax = wv.Kmax;
        tw.R_total = wv.R_total;
        tw.q0 = b->q0;
        tw.q1 = b->q1;
        tw.depth_first = c.breadth_first == 0;
        tw.ht_state = b->ht_state;
        tw.ht_key = b->ht_key;
        tw.ht_val = b->ht_val;
        tw.ht_mask = b->ht_mask;
        tw.cnt = wv.cnt;
        SBR_TRY(batch_trace_wave(tw, c.trace_blocks_per_sm, s));
        const size_t cap = (size_t)b->ht_mask + 1;
        ::sbr::note_launch(), k_batch_collect<<<nblk((int64_t)cap), 256, 0, s>>>(
            b->ht_state, b->ht_key, cap, b->nkeys + wv.j0, b->slots, c.path_cap, b->status + wv.j0);
        SBR_TRY_CUDA(cudaGetLastError());
        BatchPathArgs pa{};
        pa.jobs = jobs;
        pa.nkeys = b->nkeys + wv.j0;
        pa.slots = b->slots;
        pa.ht_key = b->ht_key;
        pa.ht_val = b->ht_val;
        pa.path_cap = c.path_cap;
        pa.raw = RefineOut{b->raw.nb, b->raw.surf, b->raw.face, b->raw.pts, b->raw.L, b->raw.aod, b->raw.aoa,
                           b->raw.ray, b->raw.dist, b->raw.jones};
        const void* rf[10] = {b->raw.nb, b->raw.surf, b->raw.face, b->raw.pts, b->raw.L, b->raw.aod, b->raw.aoa,
                              b->raw.ray, b->raw.dist, b->raw.jones};
        void* ff[10] = {b->fin.nb, b->fin.surf, b->fin.face, b->fin.pts, b->fin.L, b->fin.aod, b->fin.aoa,
                        b->fin.ray, b->fin.dist, b->fin.jones};
        const int words[10] = {1, kKmax, kKmax, 2 * 3 * kKmax, 2, 4, 4, 1, 1, 2 * kJones};
        for (int f = 0; f < 10; ++f) { pa.raw_f[f] = rf[f]; pa.fin_f[f] = ff[f]; pa.words[f] = words[f]; }
        pa.np = b->np + wv.j0;
        ::sbr::note_launch(), k_batch_paths<<<nj, kBThreads, path_smem(c.path_cap), s>>>(pa);
        SBR_TRY_CUDA(cudaGetLastError());
        BatchGainArgs ga{};
        ga.jobs = jobs;
        ga.tile_job = wv.d_tile_job;
        ga.tile_f0 = wv.d_tile_f0;
        ga.np = b->np + wv.j0;
        ga.paths = b->fin;
        ga.g = b->g;
        ga.w = b->w;
        ga.wl = b->wl;
        ga.sc = b->sc;
        ga.path_cap = synth_stride(c.path_cap);
        ::sbr::note_launch(), k_batch_gains<<<wv.n_tiles, kBThreads, 0, s>>>(ga);
        SBR_TRY_CUDA(cudaGetLastError());
        ::sbr::note_launch(), k_batch_delays<<<nj, kBThreads, 0, s>>>(jobs, b->np + wv.j0, b->fin, synth_stride(c.path_cap), b->dt, b->dr,
                                                                       b->dl);
        SBR_TRY_CUDA(cudaGetLastError());
        BatchSynthWave sw{};
        sw.jobs = jobs;
        sw.item_off = wv.d_item_off;
        sw.n_jobs = nj;
        sw.items = wv.items;
        sw.np = b->np + wv.j0;
        sw.nb = b->fin.nb;
        sw.path_cap = synth_stride(c.path_cap);
        sw.dt = b->dt;
        sw.dr = b->dr;
        sw.dl = b->dl;
        sw.w = b->w;
        sw.wl = b->wl;
        sw.sc = b->sc;
        sw.status = &wv.cnt->status;
        SBR_TRY(batch_synth_tc(sw, f16, c.tile_n, s));
        ::sbr::note_launch(), k_batch_status<<<nblk(nj), 256, 0, s>>>(wv.cnt, nj, b->status + wv.j0);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    return SBR_OK;
}

sbr_status check_job(const sbr_batch_job& j, int n_scenes, const sbr_bvh* const* scenes) {
    SBR_CHECK_ARG(j.scene >= 0 && j.scene < n_scenes, "job scene index");
    SBR_CHECK_ARG(scenes[j.scene] != nullptr && scenes[j.scene]->T >= 1, "job scene has triangles");
    SBR_CHECK_ARG(j.subdiv_N >= 1 && 10 * (int64_t)j.subdiv_N * j.subdiv_N + 2 < kBatchMaxRaysPerJob,
                  "job subdiv_N in [1, 1295]");
    SBR_CHECK_ARG(j.max_bounces >= 0 && j.max_bounces <= SBR_KMAX, "job max_bounces in [0, 8]");
    SBR_CHECK_ARG(j.pol == SBR_POL_V || j.pol == SBR_POL_H, "job pol");
    SBR_CHECK_ARG(j.F >= 1 && j.F <= 65535 && j.Nt >= 1 && j.Nr >= 1 && j.Nr <= 65535, "job F, Nt, Nr");
    SBR_CHECK_ARG(j.freqs_hz && j.tx_elem && j.rx_elem && j.H, "job device pointers");
    SBR_CHECK_ARG(std::isfinite(j.alpha) && j.alpha >= 0.0, "job alpha >= 0");
    for (int k = 0; k < 3; ++k) SBR_CHECK_ARG(std::isfinite(j.tx[k]) && std::isfinite(j.rx[k]), "job tx, rx finite");
    return SBR_OK;
}

sbr_status create(const sbr_bvh* const* scenes, const sbr_material* const* mats, int32_t n_scenes,
                  const sbr_batch_job* jobs, int32_t n_jobs, const sbr_batch_config* cfg_in, sbr_batch** out,
                  cudaStream_t s) {
    SBR_CHECK_ARG(scenes && mats && n_scenes >= 1 && jobs && n_jobs >= 1 && out, "scenes, jobs, out");
    *out = nullptr;
    for (int i = 0; i < n_scenes; ++i) SBR_CHECK_ARG(scenes[i] && mats[i], "scene handles and materials");
    for (int i = 0; i < n_jobs; ++i) SBR_TRY(check_job(jobs[i], n_scenes, scenes));
    sbr_batch_config c{};
    if (cfg_in) c = *cfg_in;
    else c.use_graph = 1;
    if (c.wave_rays == 0) c.wave_rays = (int64_t)1 << (c.breadth_first ? 26 : 28);
    if (c.path_cap == 0) c.path_cap = 512;
    if (c.tile_n == 0) c.tile_n = 128;
    if (c.precision == 0) c.precision = SBR_SYNTH_FP16X3;
    SBR_CHECK_ARG(c.path_cap >= 1 && c.path_cap <= 2048, "path_cap in [1, 2048]");
    SBR_CHECK_ARG(c.tile_n == 64 || c.tile_n == 128 || c.tile_n == 256, "tile_n in {64, 128, 256}");
    SBR_CHECK_ARG(c.precision == SBR_SYNTH_FP16X3 || c.precision == SBR_SYNTH_BF16X3, "precision");
    SBR_CHECK_ARG(c.trace_blocks_per_sm >= 0 && c.trace_blocks_per_sm <= 16, "trace_blocks_per_sm");
    SBR_CHECK_ARG(c.table_log2 == 0 || (c.table_log2 >= 4 && c.table_log2 <= 26), "table_log2");
    if (c.trace_blocks_per_sm == 0) c.trace_blocks_per_sm = batch_trace_occupancy(!c.breadth_first);
    int64_t max_R = 0;
    for (int i = 0; i < n_jobs; ++i) max_R = std::max<int64_t>(max_R, 10 * (int64_t)jobs[i].subdiv_N * jobs[i].subdiv_N + 2);
    c.wave_rays = std::max<int64_t>(c.wave_rays, max_R);

    sbr_batch* b = new (std::nothrow) sbr_batch();
    if (!b) { set_error("host allocation"); return SBR_ERR_ALLOC; }
    SBR_TRY_CUDA(cudaGetDevice(&b->device));
    b->cfg = c;
    b->n_jobs = n_jobs;
    b->jobs.assign(jobs, jobs + n_jobs);
    auto fail = [&](sbr_status st) { free_batch(b); return st; };

    // waves: jobs in order while the rays fit and the job index fits its 12 bits
    {
        Wave wv;
        wv.j0 = 0;
        for (int i = 0; i < n_jobs; ++i) {
            int64_t R = 10 * (int64_t)jobs[i].subdiv_N * jobs[i].subdiv_N + 2;
            if (i > wv.j0 && (wv.R_total + R > c.wave_rays || i - wv.j0 >= kBatchMaxJobsPerWave)) {
                wv.j1 = i;
                b->waves.push_back(wv);
                wv = Wave();
                wv.j0 = i;
            }
            wv.R_total += R;
            wv.Kmax = std::max(wv.Kmax, jobs[i].max_bounces);
            wv.seq_words += R * jobs[i].max_bounces;
        }
        wv.j1 = n_jobs;
        b->waves.push_back(wv);
    }
    int64_t max_R_wave = 0, max_seq = 0;
    for (const Wave& wv : b->waves) {
        max_R_wave = std::max(max_R_wave, wv.R_total);
        max_seq = std::max(max_seq, wv.seq_words);
        b->max_wave_jobs = std::max(b->max_wave_jobs, wv.j1 - wv.j0);
    }
    int lg = c.table_log2;
    if (lg == 0) {
        int64_t want = 2 * (int64_t)b->max_wave_jobs * c.path_cap;
        lg = 16;
        while (lg < 26 && ((int64_t)1 << lg) < want) ++lg;
        b->cfg.table_log2 = lg;
    }
    const size_t cap = (size_t)1 << lg;
    b->ht_mask = (uint32_t)(cap - 1);

    // device buffers
    sbr_status st = SBR_OK;
    if (c.breadth_first) {   // ray queues only for the breadth-first schedule
        if ((st = balloc(b, reinterpret_cast<unsigned char**>(&b->q0), (size_t)max_R_wave * 64)) != SBR_OK) return fail(st);
        if ((st = balloc(b, reinterpret_cast<unsigned char**>(&b->q1), (size_t)max_R_wave * 64)) != SBR_OK) return fail(st);
    }
    if ((st = balloc(b, &b->seq, (size_t)std::max<int64_t>(max_seq, 1))) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->ht_state, cap)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->ht_key, cap * kKeyWords)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->ht_val, cap)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->nkeys, (size_t)n_jobs)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->slots, (size_t)b->max_wave_jobs * c.path_cap)) != SBR_OK) return fail(st);
    if ((st = alloc_paths(b, &b->raw, (size_t)b->max_wave_jobs * c.path_cap)) != SBR_OK) return fail(st);
    if ((st = alloc_paths(b, &b->fin, (size_t)n_jobs * c.path_cap)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->np, (size_t)n_jobs)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->status, (size_t)n_jobs)) != SBR_OK) return fail(st);
    int64_t g_total = 0;
    b->g_base.resize(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        b->g_base[i] = g_total;
        g_total += (int64_t)c.path_cap * jobs[i].F;
    }
    if ((st = balloc(b, &b->g, (size_t)g_total)) != SBR_OK) return fail(st);

    // job records, wave tables
    std::vector<BatchJobDev> hj(n_jobs);
    int64_t max_dt = 0, max_dr = 0, max_dl = 0, max_w = 0, max_wl = 0;
    for (Wave& wv : b->waves) {
        std::vector<int64_t> ray_off, item_off;
        std::vector<int32_t> tile_job, tile_f0;
        int64_t r0 = 0, it0 = 0, sq = 0, odt = 0, odr = 0, odl = 0, ow = 0, owl = 0;
        for (int i = wv.j0; i < wv.j1; ++i) {
            const sbr_batch_job& jb = jobs[i];
            const sbr_bvh* sc = scenes[jb.scene];
            NData nd;
            if ((st = ndata(jb.subdiv_N, s, &nd)) != SBR_OK) return fail(st);
            BatchJobDev& J = hj[i];
            J = BatchJobDev{};
            J.nodes = sc->tree.nodes;
            J.tris = sc->tri_sorted;
            J.rot_stride = 3 * sc->T;
            J.plane = sc->plane_sorted;
            J.tri = sc->tri;
            J.nrm = sc->nrm;
            J.s_off = sc->s_off;
            J.s_tri = sc->s_tri;
            J.mats = mats[jb.scene];
            J.S = sc->S;
            const int64_t R = 10 * (int64_t)jb.subdiv_N * jb.subdiv_N + 2;
            J.R = (int32_t)R;
            J.K = jb.max_bounces;
            J.wave_job = i - wv.j0;
            J.geo = make_geo_n(jb.subdiv_N);
            J.seq = b->seq + sq;
            sq += R * jb.max_bounces;
            const double al = jb.alpha > 0.0 ? jb.alpha : nd.alpha;
            df a1 = df_from_double(al), a2 = df_from_double(al * al / 3.0);
            J.alpha = make_float4(a1.hi, a1.lo, a2.hi, a2.lo);
            df tx[3], rx[3];
            for (int k = 0; k < 3; ++k) {
                tx[k] = df_from_double(jb.tx[k]);
                rx[k] = df_from_double(jb.rx[k]);
                J.tx_h[k] = tx[k].hi;
                J.tx_l[k] = tx[k].lo;
                J.tx[k] = jb.tx[k];
                J.rx[k] = jb.rx[k];
            }
            J.rx_h = make_float4(rx[0].hi, rx[1].hi, rx[2].hi, 0.f);
            J.rx_l = make_float4(rx[0].lo, rx[1].lo, rx[2].lo, 0.f);
            J.F = jb.F;
            J.Nt = jb.Nt;
            J.Nr = jb.Nr;
            J.pol = jb.pol;
            J.freqs = jb.freqs_hz;
            J.gamma = jb.gamma_db_km;
            J.disp = jb.disp_deg_km;
            J.tx_elem = jb.tx_elem;
            J.rx_elem = jb.rx_elem;
            J.H = static_cast<float2*>(jb.H);
            J.path_base = (int64_t)i * c.path_cap;
            J.g_base = b->g_base[i];
            J.w_base = ow;
            ow += (int64_t)jb.F * synth_stride(c.path_cap);
            J.wl_base = owl;
            owl += jb.F;
            J.dt_base = odt;
            odt += (int64_t)synth_stride(c.path_cap) * jb.Nt;
            J.dr_base = odr;
            odr += (int64_t)synth_stride(c.path_cap) * jb.Nr;
            J.dl_base = odl;
            odl += (int64_t)jb.Nr * jb.Nt;
            ray_off.push_back(r0);
            r0 += R;
            item_off.push_back(it0);
            it0 += batch_synth_items(jb.F, jb.Nr, jb.Nt, c.tile_n);
            for (int f0 = 0; f0 < jb.F; f0 += kGainTileF) {
                tile_job.push_back(i - wv.j0);
                tile_f0.push_back(f0);
            }
        }
        ray_off.push_back(r0);
        item_off.push_back(it0);
        wv.items = it0;
        wv.n_tiles = (int)tile_job.size();
        wv.dt_words = odt; wv.dr_words = odr; wv.dl_words = odl; wv.w_words = ow;
        max_dt = std::max(max_dt, odt); max_dr = std::max(max_dr, odr);
        max_dl = std::max(max_dl, odl); max_w = std::max(max_w, ow);
        max_wl = std::max(max_wl, owl);
        if ((st = balloc(b, &wv.d_ray_off, ray_off.size())) != SBR_OK) return fail(st);
        if ((st = balloc(b, &wv.d_item_off, item_off.size())) != SBR_OK) return fail(st);
        if ((st = balloc(b, &wv.d_tile_job, tile_job.size())) != SBR_OK) return fail(st);
        if ((st = balloc(b, &wv.d_tile_f0, tile_f0.size())) != SBR_OK) return fail(st);
        if ((st = balloc(b, &wv.cnt, 1)) != SBR_OK) return fail(st);
        auto up = [&](void* d, const void* h, size_t n) -> sbr_status {
            SBR_TRY_CUDA(cudaMemcpy(d, h, n, cudaMemcpyHostToDevice));
            return SBR_OK;
        };
        if ((st = up(wv.d_ray_off, ray_off.data(), ray_off.size() * 8)) != SBR_OK) return fail(st);
        if ((st = up(wv.d_item_off, item_off.data(), item_off.size() * 8)) != SBR_OK) return fail(st);
        if ((st = up(wv.d_tile_job, tile_job.data(), tile_job.size() * 4)) != SBR_OK) return fail(st);
        if ((st = up(wv.d_tile_f0, tile_f0.data(), tile_f0.size() * 4)) != SBR_OK) return fail(st);
        b->rays += r0;
    }
    if ((st = balloc(b, &b->dt, (size_t)max_dt)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->dr, (size_t)max_dr)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->dl, (size_t)max_dl)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->w, (size_t)max_w)) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->wl, (size_t)std::max<int64_t>(1, max_wl))) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->sc, (size_t)std::max<int64_t>(1, max_wl))) != SBR_OK) return fail(st);
    if ((st = balloc(b, &b->d_jobs, (size_t)n_jobs)) != SBR_OK) return fail(st);
    if (cudaMemcpy(b->d_jobs, hj.data(), sizeof(BatchJobDev) * n_jobs, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("job table upload failed");
        return fail(SBR_ERR_CUDA);
    }
    if ((st = batch_synth_prepare(c.precision != SBR_SYNTH_BF16X3, c.tile_n)) != SBR_OK) return fail(st);
    const size_t smem = path_smem(c.path_cap);
    if (cudaFuncSetAttribute(k_batch_paths, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        set_error("path kernel shared memory %zu bytes", smem);
        return fail(SBR_ERR_CUDA);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(SBR_ERR_CUDA);
    *out = b;
    return SBR_OK;
}

sbr_status run(sbr_batch* b, cudaStream_t s) {
    if (!b->cfg.use_graph) return enqueue(b, s);
    if (!b->exec) {
        SBR_TRY_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        const long long before = sbr_launch_count();
        SBR_TRY_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        sbr_status st = enqueue(b, b->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
        const long long captured = sbr_launch_count() - before;
        note_launches(-captured);   // captured, not launched
        if (st != SBR_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) {
            set_error("stream capture failed: %s", cudaGetErrorString(e));
            return SBR_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            set_error("graph instantiation failed: %s", cudaGetErrorString(e));
            return SBR_ERR_CUDA;
        }
        b->graph_kernels = (int)captured;
    }
    SBR_TRY_CUDA(cudaGraphLaunch(b->exec, s));
    note_launches(b->graph_kernels);
    return SBR_OK;
}

}  // namespace
}  // namespace sbr

// ---------------------------------------------------------------- C ABI
using namespace sbr;

extern "C" {

sbr_status sbr_batch_create(const sbr_bvh* const* scenes, const sbr_material* const* mats, int32_t n_scenes,
                            const sbr_batch_job* jobs, int32_t n_jobs, const sbr_batch_config* cfg,
                            sbr_batch** out, void* stream) {
    clear_error();
    return create(scenes, mats, n_scenes, jobs, n_jobs, cfg, out, (cudaStream_t)stream);
}

sbr_status sbr_batch_run(sbr_batch* b, void* stream) {
    clear_error();
    SBR_CHECK_ARG(b != nullptr, "batch");
    int dev = 0;
    SBR_TRY_CUDA(cudaGetDevice(&dev));
    SBR_CHECK_ARG(dev == b->device, "current device is the batch's device");
    return run(b, (cudaStream_t)stream);
}

sbr_status sbr_batch_query(const sbr_batch* b, int32_t* n_paths, int32_t* status, sbr_batch_info* info) {
    clear_error();
    SBR_CHECK_ARG(b != nullptr, "batch");
    SBR_TRY_CUDA(cudaDeviceSynchronize());
    std::vector<int32_t> np(b->n_jobs), nk(b->n_jobs);
    std::vector<unsigned> stb(b->n_jobs);
    SBR_TRY_CUDA(cudaMemcpy(np.data(), b->np, sizeof(int32_t) * b->n_jobs, cudaMemcpyDeviceToHost));
    SBR_TRY_CUDA(cudaMemcpy(nk.data(), b->nkeys, sizeof(int32_t) * b->n_jobs, cudaMemcpyDeviceToHost));
    SBR_TRY_CUDA(cudaMemcpy(stb.data(), b->status, sizeof(unsigned) * b->n_jobs, cudaMemcpyDeviceToHost));
    int worst = SBR_OK;
    int64_t paths = 0;
    int max_keys = 0;
    for (int i = 0; i < b->n_jobs; ++i) {
        int sj = (int)status_from_bits(stb[i]);
        if (n_paths) n_paths[i] = np[i];
        if (status) status[i] = sj;
        if (sj != SBR_OK && (worst == SBR_OK || sj < worst)) worst = sj;
        paths += np[i];
        max_keys = std::max(max_keys, nk[i]);
    }
    if (worst != SBR_OK) set_error("a job of the batch failed (status %d)", worst);
    if (info) {
        memset(info, 0, sizeof *info);
        info->n_jobs = b->n_jobs;
        info->n_waves = (int32_t)b->waves.size();
        info->graph_kernels = b->graph_kernels;
        info->status = worst;
        info->max_keys = max_keys;
        info->rays = b->rays;
        info->paths = paths;
        int64_t rb = 0;
        for (const Wave& wv : b->waves) {
            TraceCountersDev c;
            SBR_TRY_CUDA(cudaMemcpy(&c, wv.cnt, sizeof c, cudaMemcpyDeviceToHost));
            for (int k = 0; k <= wv.Kmax; ++k) rb += (int64_t)c.queue[k];
        }
        info->ray_bounces = rb;
        info->config = b->cfg;
    }
    return (sbr_status)worst;
}

sbr_status sbr_batch_export(const sbr_batch* b, int32_t job, int32_t n, int32_t* n_bounce, int32_t* surf_seq,
                            int32_t* face_seq, double* pts, double* length, double* aod, double* aoa,
                            uint32_t* ray_id, float* dist, void* gains, void* stream) {
    clear_error();
    SBR_CHECK_ARG(b != nullptr && job >= 0 && job < b->n_jobs, "batch and job");
    SBR_CHECK_ARG(n >= 0 && n <= b->cfg.path_cap, "n <= path_cap");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t o = (int64_t)job * b->cfg.path_cap;
    auto cp = [&](void* dst, const void* src, size_t bytes) -> sbr_status {
        if (!dst || bytes == 0) return SBR_OK;
        SBR_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
        return SBR_OK;
    };
    SBR_TRY(cp(n_bounce, b->fin.nb + o, sizeof(int32_t) * n));
    SBR_TRY(cp(surf_seq, b->fin.surf + o * kKmax, sizeof(int32_t) * n * kKmax));
    SBR_TRY(cp(face_seq, b->fin.face + o * kKmax, sizeof(int32_t) * n * kKmax));
    SBR_TRY(cp(pts, b->fin.pts + o * kKmax * 3, sizeof(double) * n * kKmax * 3));
    SBR_TRY(cp(length, b->fin.L + o, sizeof(double) * n));
    SBR_TRY(cp(aod, b->fin.aod + o * 2, sizeof(double) * n * 2));
    SBR_TRY(cp(aoa, b->fin.aoa + o * 2, sizeof(double) * n * 2));
    SBR_TRY(cp(ray_id, b->fin.ray + o, sizeof(uint32_t) * n));
    SBR_TRY(cp(dist, b->fin.dist + o, sizeof(float) * n));
    SBR_TRY(cp(gains, b->g + b->g_base[job], sizeof(float2) * (size_t)n * b->jobs[job].F));
    return SBR_OK;
}

void sbr_batch_free(sbr_batch* b) { free_batch(b); }

sbr_status sbr_batch_tune(const sbr_bvh* const* scenes, const sbr_material* const* mats, int32_t n_scenes,
                          const sbr_batch_job* jobs, int32_t n_jobs, sbr_batch_config* cfg, double* ms,
                          void* stream) {
    clear_error();
    SBR_CHECK_ARG(cfg != nullptr, "cfg");
    cudaStream_t s = (cudaStream_t)stream;
    const sbr_batch_config fixed = *cfg;
    sbr_batch_config best = fixed;
    if (best.use_graph == 0) best.use_graph = 1;
    // one candidate: create, two warm runs, median of three timed runs
    auto time_cfg = [&](sbr_batch_config c, double* t_ms, int* max_keys, sbr_batch_config* resolved) -> sbr_status {
        sbr_batch* b = nullptr;
        SBR_TRY(create(scenes, mats, n_scenes, jobs, n_jobs, &c, &b, s));
        sbr_status st = SBR_OK;
        for (int k = 0; k < 2 && st == SBR_OK; ++k) st = run(b, s);
        std::vector<float> ts;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (st == SBR_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = SBR_ERR_CUDA;
        for (int k = 0; k < 3 && st == SBR_OK; ++k) {
            cudaEventRecord(e0, s);
            st = run(b, s);
            cudaEventRecord(e1, s);
            float t = 0.f;
            if (st == SBR_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
                ts.push_back(t);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        sbr_batch_info info{};
        sbr_status q = st == SBR_OK ? sbr_batch_query(b, nullptr, nullptr, &info) : st;
        free_batch(b);
        if (st != SBR_OK) return st;
        if (q != SBR_OK && q != SBR_ERR_CAPACITY) return q;
        if (ts.empty()) { set_error("timing failed"); return SBR_ERR_CUDA; }
        std::sort(ts.begin(), ts.end());
        *t_ms = ts[ts.size() / 2];
        *max_keys = info.max_keys;
        *resolved = info.config;   // defaults made explicit
        return SBR_OK;
    };
    double t = 0;
    int mk = 0;
    sbr_batch_config res{};
    // path store: a first run at the given (or 1024) capacity sizes it to the keys seen
    if (fixed.path_cap == 0) {
        sbr_batch_config c = best;
        c.path_cap = 1024;
        SBR_TRY(time_cfg(c, &t, &mk, &res));
        int cap = 64;
        while (cap < 2048 && cap < (int)std::ceil(1.5 * mk)) cap <<= 1;
        best.path_cap = cap;
    }
    double best_t = 1e300;
    // coordinate search: tile width, then bounce grid, then ray-queue capacity
    const int tiles[3] = {64, 128, 256};
    // resident blocks per SM of the trace kernel: all of them, three quarters, half
    const int occ = batch_trace_occupancy(!fixed.breadth_first);
    const int grids[3] = {occ, std::max(1, (3 * occ) / 4), std::max(1, occ / 2)};
    const int sh = fixed.breadth_first ? 25 : 26;
    const int64_t waves[3] = {(int64_t)1 << sh, (int64_t)1 << (sh + 1), (int64_t)1 << (sh + 2)};
    auto consider = [&](sbr_batch_config c) -> sbr_status {
        SBR_TRY(time_cfg(c, &t, &mk, &res));
        if (t < best_t) { best_t = t; best = res; }
        return SBR_OK;
    };
    if (fixed.tile_n == 0) {
        for (int tn : tiles) { sbr_batch_config c = best; c.tile_n = tn; SBR_TRY(consider(c)); }
    } else {
        SBR_TRY(consider(best));
    }
    if (fixed.trace_blocks_per_sm == 0) {
        sbr_batch_config base = best;
        for (int g : grids) { sbr_batch_config c = base; c.trace_blocks_per_sm = g; SBR_TRY(consider(c)); }
    }
    if (fixed.wave_rays == 0) {
        sbr_batch_config base = best;
        for (int64_t wr : waves) { sbr_batch_config c = base; c.wave_rays = wr; SBR_TRY(consider(c)); }
    }
    *cfg = best;
    if (ms) *ms = best_t;
    return SBR_OK;
}

}  // extern "C"
