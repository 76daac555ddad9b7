// C ABI of libsbr (include/sbr.h): host-side validation, handle lifetime and
// dispatch to the kernels of the other translation units.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>

#include "sbr_internal.cuh"

namespace sbr {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

sbr_status status_from_bits(uint32_t bits) {
    if (bits & ST_CAPACITY) { set_error("device dedup table full"); return SBR_ERR_CAPACITY; }
    if (bits & ST_STACK) { set_error("BVH traversal stack overflow"); return SBR_ERR_STACK_OVERFLOW; }
    if (bits & ST_TIMEOUT) { set_error("bounded device wait gave up"); return SBR_ERR_TIMEOUT; }
    if (bits & ST_NUMERIC) { set_error("non-finite value on the device"); return SBR_ERR_NUMERIC; }
    return SBR_OK;
}

// The stream-ordered pool of each device keeps freed blocks instead of returning
// them to the CUDA driver at every synchronisation (its default), so that the
// buffers of consecutive calls reuse the same memory.
static void keep_pool_memory() {
    static std::mutex mu;
    static bool done[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

// Host-driven fault injection for tests (SBR_FAULT environment variable, read
// at each use): "alloc" makes every library allocation fail; "timeout" makes
// the tensor-core synthesis wait on a barrier nothing arrives at, with a short
// bound, so that it reports SBR_ERR_TIMEOUT. No injected fault touches the GPU
// beyond a bounded wait.
int fault_mode() {
    const char* e = getenv("SBR_FAULT");
    if (!e) return kFaultNone;
    if (!strcmp(e, "alloc")) return kFaultAlloc;
    if (!strcmp(e, "timeout")) return kFaultTimeout;
    return kFaultNone;
}

sbr_status dalloc(void** p, size_t bytes, cudaStream_t s) {
    if (fault_mode() == kFaultAlloc) {
        *p = nullptr;
        set_error("injected allocation failure (SBR_FAULT=alloc), %zu bytes", bytes);
        return SBR_ERR_ALLOC;
    }
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return SBR_ERR_ALLOC;
    }
    return SBR_OK;
}

void dfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

namespace {
__global__ void k_set_u64(unsigned long long* dst, unsigned long long v) { *dst = v; }
}  // namespace

sbr_status set_u64(unsigned long long* dst, unsigned long long v, cudaStream_t s) {
    ::sbr::note_launch(), k_set_u64<<<1, 1, 0, s>>>(dst, v);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}


static int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

static bool finite3(const double* v) {
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

}  // namespace sbr

using namespace sbr;

#define SBR_SAME_DEVICE(h)                                                        \
    do {                                                                          \
        if ((h)->device != current_device()) {                                    \
            set_error("handle used on a device other than the one it was made on"); \
            return SBR_ERR_INVALID_ARG;                                           \
        }                                                                         \
    } while (0)

extern "C" {

const char* sbr_last_error(void) { return g_err; }

const char* sbr_version(void) { return "sbr-gb300 0.1 (sm_103a)"; }

int64_t sbr_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

sbr_status sbr_launch_dirs(int32_t N, double* dirs, double* alpha, void* stream) {
    clear_error();
    SBR_CHECK_ARG(N >= 1 && N <= 20000, "N in [1, 20000]");
    SBR_CHECK_ARG(dirs != nullptr || alpha != nullptr, "dirs or alpha");
    cudaStream_t s = (cudaStream_t)stream;
    if (dirs) SBR_TRY(launch_dirs(N, dirs, s));
    if (alpha) SBR_TRY(launch_alpha(N, alpha, s));
    return SBR_OK;
}

sbr_status sbr_build_bvh(const float* tri_xyz, const int32_t* surface_id, int64_t T, int32_t S,
                         sbr_bvh** out, void* stream) {
    return sbr_build_bvh_ex(tri_xyz, surface_id, T, S, 0u, out, stream);
}

sbr_status sbr_build_bvh_ex(const float* tri_xyz, const int32_t* surface_id, int64_t T, int32_t S,
                            uint32_t flags, sbr_bvh** out, void* stream) {
    clear_error();
    SBR_CHECK_ARG(out != nullptr, "out");
    *out = nullptr;
    SBR_CHECK_ARG((flags & ~(uint32_t)SBR_BVH_SAH_TOP) == 0, "flags: SBR_BVH_SAH_TOP only");
    *out = nullptr;
    SBR_CHECK_ARG(T >= 0 && T < ((int64_t)1 << 28), "0 <= T < 2^28");
    SBR_CHECK_ARG(S >= 0 && (T == 0 || S >= 1), "S >= 1 when T > 0");
    SBR_CHECK_ARG(T == 0 || (tri_xyz && surface_id), "tri_xyz and surface_id");
    cudaStream_t s = (cudaStream_t)stream;
    sbr_bvh* b = new (std::nothrow) sbr_bvh();
    if (!b) { set_error("host allocation failed"); return SBR_ERR_ALLOC; }
    b->device = current_device();
    b->stream = s;
    sbr_status st = bvh_build(tri_xyz, surface_id, T, S, b, s, (flags & SBR_BVH_SAH_TOP) != 0);
    if (st != SBR_OK) {
        sbr_bvh_free(b);
        return st;
    }
    *out = b;
    return SBR_OK;
}

void sbr_bvh_free(sbr_bvh* b) {
    if (!b) return;
    cudaStream_t s = b->stream;
    free_lbvh(&b->tree, s);
    dfree(b->tri_rot, s); dfree(b->plane_sorted, s); dfree(b->tri, s); dfree(b->surf, s);
    dfree(b->nrm, s); dfree(b->s_off, s); dfree(b->s_tri, s); dfree(b->d_depth, s);
    delete b;
}

sbr_status sbr_bvh_query(const sbr_bvh* b, sbr_bvh_info* out) {
    clear_error();
    SBR_CHECK_ARG(b && out, "bvh and out");
    SBR_SAME_DEVICE(b);
    int32_t depth = 0;
    SBR_TRY_CUDA(cudaMemcpyAsync(&depth, b->d_depth, sizeof depth, cudaMemcpyDeviceToHost, b->stream));
    SBR_TRY_CUDA(cudaStreamSynchronize(b->stream));
    out->T = b->T;
    out->S = b->S;
    out->n_nodes = b->tree.n_nodes;
    out->depth = depth;
    out->reserved = 0;
    return SBR_OK;
}

sbr_status sbr_trace(const sbr_bvh* b, const sbr_trace_params* p, sbr_trace_result** out,
                     void* stream) {
    clear_error();
    SBR_CHECK_ARG(out != nullptr, "out");
    *out = nullptr;
    SBR_CHECK_ARG(b && p, "bvh and params");
    SBR_SAME_DEVICE(b);
    SBR_CHECK_ARG(p->subdiv_N >= 1 && p->subdiv_N <= 20000, "subdiv_N in [1, 20000]");
    SBR_CHECK_ARG(p->max_bounces >= 0 && p->max_bounces <= SBR_KMAX, "max_bounces in [0, 8]");
    SBR_CHECK_ARG(p->n_rx >= 0 && p->n_rx <= (1 << 20), "n_rx in [0, 2^20]");
    SBR_CHECK_ARG(p->n_rx == 0 || p->rx_xyz, "rx_xyz");
    SBR_CHECK_ARG(finite3(p->tx), "finite tx");
    SBR_CHECK_ARG(std::isfinite(p->alpha) && p->alpha >= 0.0, "alpha >= 0");
    SBR_CHECK_ARG(p->table_log2 == 0 || (p->table_log2 >= 4 && p->table_log2 <= 28), "table_log2");
    SBR_CHECK_ARG(p->depth_first_from >= 0, "depth_first_from >= 0");
    int64_t R = 10 * (int64_t)p->subdiv_N * p->subdiv_N + 2;
    SBR_CHECK_ARG(R < ((int64_t)1 << 32), "10 N^2 + 2 < 2^32");
    const int64_t ray_end = p->ray_end ? p->ray_end : R;
    SBR_CHECK_ARG(p->ray_begin >= 0 && p->ray_begin < ray_end && ray_end <= R,
                  "0 <= ray_begin < ray_end <= 10 N^2 + 2");
    cudaStream_t s = (cudaStream_t)stream;
    sbr_trace_result* tr = new (std::nothrow) sbr_trace_result();
    if (!tr) { set_error("host allocation failed"); return SBR_ERR_ALLOC; }
    tr->device = current_device();
    tr->stream = s;
    tr->params = *p;
    tr->R = R;
    tr->ray0 = p->ray_begin;
    tr->Rr = ray_end - p->ray_begin;
    tr->n_rx = p->n_rx;
    tr->df_from = p->depth_first_from;
    if (p->table_log2) {
        tr->table_log2 = p->table_log2;
    } else {
        int lg = 14;
        while (lg < 26 && ((int64_t)1 << lg) < (int64_t)p->n_rx * 512) ++lg;
        tr->table_log2 = lg;
    }
    sbr_status st = SBR_OK;
    if (tr->n_rx > 0) {
        st = dalloc_n(&tr->rx, 3 * (size_t)tr->n_rx, s);
        if (st == SBR_OK &&
            cudaMemcpyAsync(tr->rx, p->rx_xyz, sizeof(double) * 3 * tr->n_rx, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess) {
            set_error("copy of rx_xyz failed");
            st = SBR_ERR_CUDA;
        }
    }
    if (st == SBR_OK) st = dalloc_n(&tr->d_alpha, 1, s);
    // a given alpha is stored by the trace's set-up launch; the default one
    // (alpha = 0) is computed from the launch grid first
    if (st == SBR_OK && !(p->alpha > 0.0)) st = launch_alpha_fast(p->subdiv_N, tr->d_alpha, s);
    if (st == SBR_OK) st = trace_run(b, tr, s);
    if (st != SBR_OK) {
        sbr_trace_free(tr);
        return st;
    }
    *out = tr;
    return SBR_OK;
}

sbr_status sbr_trace_stats(const sbr_trace_result* tr, sbr_trace_counters* out) {
    clear_error();
    SBR_CHECK_ARG(tr && out, "trace result and out");
    SBR_SAME_DEVICE(tr);
    TraceCountersDev c;
    double alpha = 0;
    if (tr->h_valid) {   // final counters already on the host (taken when the path list was built)
        c = tr->h_cnt;
        alpha = tr->h_alpha;
    } else {
        SBR_TRY_CUDA(cudaMemcpyAsync(&c, tr->cnt, sizeof c, cudaMemcpyDeviceToHost, tr->stream));
        SBR_TRY_CUDA(cudaMemcpyAsync(&alpha, tr->d_alpha, sizeof alpha, cudaMemcpyDeviceToHost, tr->stream));
        SBR_TRY_CUDA(cudaStreamSynchronize(tr->stream));
    }
    memset(out, 0, sizeof *out);
    out->rays = tr->Rr;
    int64_t rb = 0;
    for (int k = 0; k <= tr->params.max_bounces; ++k) rb += (int64_t)c.queue[k];
    out->ray_bounces = rb;
    out->candidates = (int64_t)c.candidates;
    out->keys = (int64_t)c.keys;
    out->fp64_segments = (int64_t)c.fp64_segments;
    out->fp64_tests = (int64_t)c.fp64_tests;
    out->node_visits = (int64_t)c.node_visits;
    out->tri_tests = (int64_t)c.tri_tests;
    out->rx_visits = (int64_t)c.rx_visits;
    out->near_edge_hits = (int64_t)c.near_edge_hits;
    for (int k = 0; k < SBR_KMAX + 2; ++k) out->queue[k] = (int64_t)c.queue[k];
    out->alpha = alpha;
    out->table_log2 = tr->table_log2;
    if (tr->ev[0]) {
        for (int k = 0; k <= tr->params.max_bounces; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, tr->ev[k], tr->ev[k + 1]) == cudaSuccess) out->bounce_ms[k] = ms;
        }
    }
    out->status = (int32_t)status_from_bits(c.status);
    return (sbr_status)out->status;
}

sbr_status sbr_trace_entries(const sbr_trace_result* tr, uint32_t* keys, uint64_t* vals, int64_t cap,
                             int64_t* n_out, void* stream) {
    clear_error();
    SBR_CHECK_ARG(tr && n_out, "trace result and n_out");
    SBR_CHECK_ARG(cap >= 0 && (cap == 0 || (keys && vals)), "cap >= 0, keys and vals");
    SBR_SAME_DEVICE(tr);
    *n_out = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (tr->stream != s) SBR_TRY_CUDA(cudaStreamSynchronize(tr->stream));
    return trace_entries_run(tr, keys, reinterpret_cast<unsigned long long*>(vals), cap, n_out, s);
}

sbr_status sbr_trace_merge(const sbr_trace_params* p, const uint32_t* keys, const uint64_t* vals, int64_t n,
                           sbr_trace_result** out, void* stream) {
    clear_error();
    SBR_CHECK_ARG(out != nullptr, "out");
    *out = nullptr;
    SBR_CHECK_ARG(p != nullptr, "params");
    SBR_CHECK_ARG(n >= 0 && (n == 0 || (keys && vals)), "n >= 0, keys and vals");
    SBR_CHECK_ARG(p->subdiv_N >= 1 && p->subdiv_N <= 20000, "subdiv_N in [1, 20000]");
    SBR_CHECK_ARG(p->max_bounces >= 0 && p->max_bounces <= SBR_KMAX, "max_bounces in [0, 8]");
    SBR_CHECK_ARG(p->n_rx >= 0 && p->n_rx <= (1 << 20), "n_rx in [0, 2^20]");
    SBR_CHECK_ARG(p->n_rx == 0 || p->rx_xyz, "rx_xyz");
    SBR_CHECK_ARG(finite3(p->tx), "finite tx");
    SBR_CHECK_ARG(std::isfinite(p->alpha) && p->alpha >= 0.0, "alpha >= 0");
    SBR_CHECK_ARG(p->table_log2 == 0 || (p->table_log2 >= 4 && p->table_log2 <= 28), "table_log2");
    cudaStream_t s = (cudaStream_t)stream;
    sbr_trace_result* tr = new (std::nothrow) sbr_trace_result();
    if (!tr) { set_error("host allocation failed"); return SBR_ERR_ALLOC; }
    tr->device = current_device();
    tr->stream = s;
    tr->params = *p;
    tr->R = 10 * (int64_t)p->subdiv_N * p->subdiv_N + 2;
    tr->ray0 = 0;
    tr->Rr = 0;   // no ray is traced by the merge itself
    tr->n_rx = p->n_rx;
    tr->df_from = 0;
    if (p->table_log2) {
        tr->table_log2 = p->table_log2;
    } else {
        int lg = 10;
        while (lg < 28 && ((int64_t)1 << lg) < 2 * n) ++lg;   // load factor <= 1/2
        tr->table_log2 = lg;
    }
    sbr_status st = SBR_OK;
    if (tr->n_rx > 0) {
        st = dalloc_n(&tr->rx, 3 * (size_t)tr->n_rx, s);
        if (st == SBR_OK &&
            cudaMemcpyAsync(tr->rx, p->rx_xyz, sizeof(double) * 3 * tr->n_rx, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess) {
            set_error("copy of rx_xyz failed");
            st = SBR_ERR_CUDA;
        }
    }
    if (st == SBR_OK) st = dalloc_n(&tr->d_alpha, 1, s);
    if (st == SBR_OK && !(p->alpha > 0.0)) st = launch_alpha_fast(p->subdiv_N, tr->d_alpha, s);
    if (st == SBR_OK) st = trace_merge_run(tr, keys, reinterpret_cast<const unsigned long long*>(vals), n, s);
    if (st != SBR_OK) {
        sbr_trace_free(tr);
        return st;
    }
    *out = tr;
    return SBR_OK;
}

void sbr_trace_free(sbr_trace_result* tr) {
    if (!tr) return;
    cudaStream_t s = tr->stream;
    dfree(tr->seqf, s); dfree(tr->rx, s); dfree(tr->d_alpha, s); dfree(tr->ht_state, s); dfree(tr->ht_key, s);
    dfree(tr->ht_val, s); dfree(tr->cnt, s);
    for (auto& e : tr->ev)
        if (e) cudaEventDestroy(e);
    delete tr;
}

sbr_status sbr_paths(const sbr_trace_result* tr, const sbr_bvh* b, sbr_path_list** out,
                     int64_t* n_paths_out, void* stream) {
    clear_error();
    SBR_CHECK_ARG(out != nullptr, "out");
    *out = nullptr;
    SBR_CHECK_ARG(tr && b, "trace result and bvh");
    SBR_SAME_DEVICE(tr);
    SBR_SAME_DEVICE(b);
    cudaStream_t s = (cudaStream_t)stream;
    // the trace must have finished cleanly before its table is read. On the
    // trace's own stream the path kernels are ordered after it and its status
    // is read together with the key count (paths_run's first wait); on another
    // stream the host waits for the trace here
    if (tr->stream != s) {
        unsigned bits = 0;
        SBR_TRY_CUDA(cudaMemcpyAsync(&bits, &tr->cnt->status, sizeof bits, cudaMemcpyDeviceToHost, tr->stream));
        SBR_TRY_CUDA(cudaStreamSynchronize(tr->stream));
        SBR_TRY(status_from_bits(bits));
    }
    sbr_path_list* pl = new (std::nothrow) sbr_path_list();
    if (!pl) { set_error("host allocation failed"); return SBR_ERR_ALLOC; }
    pl->device = current_device();
    pl->stream = s;
    pl->S = b->S;
    sbr_status st = paths_run(tr, b, pl, s);
    if (st != SBR_OK) {
        sbr_path_list_free(pl);
        return st;
    }
    *out = pl;
    if (n_paths_out) *n_paths_out = pl->P;
    return SBR_OK;
}

sbr_status sbr_path_query(const sbr_path_list* pl, sbr_path_info* out) {
    clear_error();
    SBR_CHECK_ARG(pl && out, "path list and out");
    SBR_SAME_DEVICE(pl);
    unsigned bits = 0;
    SBR_TRY_CUDA(cudaMemcpyAsync(&bits, pl->d_status, sizeof bits, cudaMemcpyDeviceToHost, pl->stream));
    SBR_TRY_CUDA(cudaStreamSynchronize(pl->stream));
    out->n_paths = pl->P;
    out->n_keys = pl->n_keys;
    out->n_invalid = pl->n_invalid;
    out->n_rx = pl->n_rx;
    out->max_bounces = pl->K;
    out->status = (int32_t)status_from_bits(bits);
    out->reserved = 0;
    return (sbr_status)out->status;
}

sbr_status sbr_path_export(const sbr_path_list* pl, int32_t* rx, int32_t* n_bounce, int32_t* surf_seq,
                           int32_t* face_seq, double* pts, double* length, double* aod, double* aoa,
                           uint32_t* ray_id, float* dist, void* stream) {
    clear_error();
    SBR_CHECK_ARG(pl != nullptr, "path list");
    SBR_SAME_DEVICE(pl);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t P = (size_t)pl->P;
    if (P == 0) return SBR_OK;
    auto cp = [&](void* dst, const void* src, size_t bytes) -> sbr_status {
        if (!dst) return SBR_OK;
        // device or (pinned) host destination, resolved by unified addressing
        SBR_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
        return SBR_OK;
    };
    SBR_TRY(cp(rx, pl->rx, P * sizeof(int32_t)));
    SBR_TRY(cp(n_bounce, pl->nb, P * sizeof(int32_t)));
    SBR_TRY(cp(surf_seq, pl->surf, P * kKmax * sizeof(int32_t)));
    SBR_TRY(cp(face_seq, pl->face, P * kKmax * sizeof(int32_t)));
    SBR_TRY(cp(pts, pl->pts, P * kKmax * 3 * sizeof(double)));
    SBR_TRY(cp(length, pl->L, P * sizeof(double)));
    SBR_TRY(cp(aod, pl->aod, P * 2 * sizeof(double)));
    SBR_TRY(cp(aoa, pl->aoa, P * 2 * sizeof(double)));
    SBR_TRY(cp(ray_id, pl->ray, P * sizeof(uint32_t)));
    SBR_TRY(cp(dist, pl->dist, P * sizeof(float)));
    return SBR_OK;
}

void sbr_path_list_free(sbr_path_list* pl) {
    if (!pl) return;
    cudaStream_t s = pl->stream;
    dfree(pl->rx_xyz, s); dfree(pl->rx, s); dfree(pl->nb, s); dfree(pl->surf, s); dfree(pl->face, s);
    dfree(pl->pts, s); dfree(pl->L, s); dfree(pl->aod, s); dfree(pl->aoa, s); dfree(pl->ray, s);
    dfree(pl->dist, s); dfree(pl->jones, s); dfree(pl->rx_off, s); dfree(pl->d_status, s);
    delete[] pl->h_rx_off;
    delete pl;
}

sbr_status sbr_path_gains(const sbr_path_list* pl, const sbr_material* mats, int32_t S,
                          const double* freqs_hz, int32_t F, const float* gamma_db_km,
                          const float* disp_deg_km, int32_t pol, void* gains, void* stream) {
    clear_error();
    SBR_CHECK_ARG(pl != nullptr, "path list");
    SBR_SAME_DEVICE(pl);
    SBR_CHECK_ARG(F >= 1, "F >= 1");
    SBR_CHECK_ARG(freqs_hz && (gains || pl->P == 0), "freqs_hz and gains (gains may be NULL without paths)");
    SBR_CHECK_ARG(S >= pl->S, "materials for every surface id of the scene");
    SBR_CHECK_ARG(pl->P == 0 || pl->S == 0 || mats, "mats");
    SBR_CHECK_ARG(pol == SBR_POL_V || pol == SBR_POL_H, "pol");
    return gains_run(pl, mats, S, freqs_hz, F, gamma_db_km, disp_deg_km, pol, (float2*)gains,
                     (cudaStream_t)stream);
}

sbr_status sbr_synthesize_H(const sbr_path_list* pl, const void* gains, const double* freqs_hz,
                            int32_t F, const double* tx_elem, int32_t Nt, const double* rx_elem,
                            int32_t Nr, int32_t rx_index, int32_t precision, void* H, void* stream) {
    clear_error();
    SBR_CHECK_ARG(pl != nullptr, "path list");
    SBR_SAME_DEVICE(pl);
    SBR_CHECK_ARG(F >= 1 && Nt >= 1 && Nr >= 1, "F, Nt, Nr >= 1");
    SBR_CHECK_ARG(F <= 65535 && Nr <= 65535, "F, Nr <= 65535");
    SBR_CHECK_ARG((gains || pl->P == 0) && freqs_hz && tx_elem && rx_elem && H, "pointers (gains may be NULL without paths)");
    SBR_CHECK_ARG(rx_index >= 0 && rx_index < pl->n_rx, "rx_index");
    cudaStream_t s = (cudaStream_t)stream;
    switch (precision) {
        case SBR_SYNTH_FP64:
        case SBR_SYNTH_FP32:
            return synth_simt_run(pl, (const float2*)gains, freqs_hz, F, tx_elem, Nt, rx_elem, Nr,
                                  rx_index, precision == SBR_SYNTH_FP64, (float2*)H, s);
        case SBR_SYNTH_BF16X3:
        case SBR_SYNTH_FP16X3:
            return synth_tc_run(pl, (const float2*)gains, freqs_hz, F, tx_elem, Nt, rx_elem, Nr,
                                rx_index, (float2*)H, precision == SBR_SYNTH_FP16X3, s);
        default:
            set_error("unknown precision %d", precision);
            return SBR_ERR_INVALID_ARG;
    }
}

sbr_status sbr_synthesize_H_elements(const sbr_path_list* pl, const void* gains, const double* freqs_hz,
                                     int32_t F, const double* tx_elem, int32_t Nt, int32_t precision,
                                     void* H, void* stream) {
    clear_error();
    SBR_CHECK_ARG(pl != nullptr, "path list");
    SBR_SAME_DEVICE(pl);
    SBR_CHECK_ARG(F >= 1 && Nt >= 1, "F, Nt >= 1");
    SBR_CHECK_ARG(F <= 65535 && pl->n_rx >= 1 && pl->n_rx <= 65535, "F <= 65535, 1 <= n_rx <= 65535");
    SBR_CHECK_ARG(pl->P <= INT32_MAX, "P < 2^31");
    SBR_CHECK_ARG((gains || pl->P == 0) && freqs_hz && tx_elem && H, "pointers (gains may be NULL without paths)");
    SBR_CHECK_ARG(precision == SBR_SYNTH_FP64 || precision == SBR_SYNTH_FP32, "precision FP64 or FP32");
    return synth_elements_run(pl, (const float2*)gains, freqs_hz, F, tx_elem, Nt, precision == SBR_SYNTH_FP64,
                              (float2*)H, (cudaStream_t)stream);
}

sbr_status sbr_pdp_angles(const sbr_path_list* pl, const void* gains, int32_t F, int32_t f_index,
                          double fc_hz, double bin_s, int32_t n_bins, float* pdp_db, double* stats,
                          void* stream) {
    clear_error();
    SBR_CHECK_ARG(pl != nullptr, "path list");
    SBR_SAME_DEVICE(pl);
    SBR_CHECK_ARG(F >= 1 && f_index >= 0 && f_index < F, "f_index in [0, F)");
    SBR_CHECK_ARG(bin_s > 0 && std::isfinite(bin_s) && std::isfinite(fc_hz), "bin_s > 0, finite fc");
    SBR_CHECK_ARG(n_bins >= 1 && n_bins <= 16384, "n_bins in [1, 16384]");
    SBR_CHECK_ARG(pl->n_rx == 0 || (pdp_db && stats), "pdp_db and stats");
    SBR_CHECK_ARG(pl->P == 0 || gains, "gains");
    return pdp_run(pl, (const float2*)gains, F, f_index, fc_hz, bin_s, n_bins, pdp_db, stats,
                   (cudaStream_t)stream);
}

sbr_status sbr_surrogate_targets(const sbr_path_list* pl, const void* gains, int32_t F, int32_t n_taps,
                                 double tap_s, double floor_db, float* out, void* stream) {
    clear_error();
    SBR_CHECK_ARG(pl != nullptr, "path list");
    SBR_SAME_DEVICE(pl);
    SBR_CHECK_ARG(F >= 1 && n_taps >= 1 && n_taps <= 32, "F >= 1, n_taps in [1, 32]");
    SBR_CHECK_ARG(tap_s > 0 && std::isfinite(tap_s) && std::isfinite(floor_db), "tap_s > 0, finite floor_db");
    SBR_CHECK_ARG(pl->n_rx == 0 || out, "out");
    SBR_CHECK_ARG(pl->P == 0 || gains, "gains");
    return surrogate_targets_run(pl, (const float2*)gains, F, n_taps, tap_s, floor_db, out, (cudaStream_t)stream);
}

sbr_status sbr_capacity(const void* H, int32_t F, int32_t Nr, int32_t Nt, const double* snr_db,
                        int32_t n_snr, double* C, void* stream) {
    clear_error();
    SBR_CHECK_ARG(H && snr_db && C, "pointers");
    SBR_CHECK_ARG(F >= 1 && Nr >= 1 && Nt >= 1, "F, Nr, Nt >= 1");
    SBR_CHECK_ARG((Nr < Nt ? Nr : Nt) <= 64, "min(Nr, Nt) <= 64");
    SBR_CHECK_ARG(n_snr >= 1 && n_snr <= 32, "n_snr in [1, 32]");
    for (int i = 0; i < n_snr; ++i) SBR_CHECK_ARG(std::isfinite(snr_db[i]), "finite snr_db");
    return capacity_run((const float2*)H, F, Nr, Nt, snr_db, n_snr, C, (cudaStream_t)stream);
}

sbr_status sbr_capacity_noalloc(const void* H, int32_t F, int32_t Nr, int32_t Nt, const double* snr_db,
                                int32_t n_snr, double* C, void* stream) {
    clear_error();
    SBR_CHECK_ARG(H && snr_db && C, "pointers");
    SBR_CHECK_ARG(F >= 1 && Nr >= 1 && Nt >= 1, "F, Nr, Nt >= 1");
    SBR_CHECK_ARG((Nr < Nt ? Nr : Nt) <= 64, "min(Nr, Nt) <= 64");
    SBR_CHECK_ARG(n_snr >= 1, "n_snr >= 1");
    for (int i = 0; i < n_snr; ++i) SBR_CHECK_ARG(std::isfinite(snr_db[i]), "finite snr_db");
    return capacity_noalloc_run((const float2*)H, F, Nr, Nt, snr_db, n_snr, C, (cudaStream_t)stream);
}

}  // extern "C"
