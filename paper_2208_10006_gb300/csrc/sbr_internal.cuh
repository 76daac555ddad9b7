// Internal declarations shared by the CUDA translation units of libsbr.
// Not part of the public ABI (include/sbr.h).
#pragma once
#include <atomic>
#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbr.h"

namespace sbr {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();

#define SBR_TRY_CUDA(expr)                                                             \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::sbr::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),   \
                             __FILE__, __LINE__);                                      \
            return SBR_ERR_CUDA;                                                       \
        }                                                                              \
    } while (0)

#define SBR_TRY(expr)                      \
    do {                                   \
        sbr_status s_ = (expr);            \
        if (s_ != SBR_OK) return s_;       \
    } while (0)

#define SBR_CHECK_ARG(cond, msg)                                          \
    do {                                                                  \
        if (!(cond)) {                                                    \
            ::sbr::set_error("invalid argument: %s (%s)", msg, #cond);    \
            return SBR_ERR_INVALID_ARG;                                   \
        }                                                             \
    } while (0)

// device status word bits (written with atomicOr, read by synchronous calls)
enum : uint32_t {
    ST_CAPACITY = 1u,
    ST_STACK = 2u,
    ST_TIMEOUT = 4u,
    ST_NUMERIC = 8u,
};
sbr_status status_from_bits(uint32_t bits);

constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;
constexpr int kKmax = SBR_KMAX;
constexpr int kKeyWords = 2 + kKmax;  // rx, n_bounce, surface sequence

// stream-ordered allocation helpers
sbr_status dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);
template <class T>
sbr_status dalloc_n(T** p, size_t n, cudaStream_t s) {
    return dalloc(reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? 16 : 0), s);
}
int sm_count();
// a kernel's dynamic shared-memory limit, set once per device (the attribute
// belongs to the current device's context); devmask holds the devices done
inline sbr_status set_smem_once(const void* func, int bytes, std::atomic<unsigned long long>* devmask) {
    int dev = 0;
    SBR_TRY_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (devmask->load() & bit)) return SBR_OK;
    SBR_TRY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    if (bit) devmask->fetch_or(bit);
    return SBR_OK;
}
// count of kernel launches made by the library in this process
void note_launch();
// Programmatic dependent launch: the kernel may be scheduled while its
// predecessor on the stream finishes (its launch latency overlaps that tail);
// every kernel launched this way calls pdl_wait() before its first memory
// access, which returns once the predecessor has completed and its writes are
// visible, so the stream order is kept (pdl_wait is a no-op for an ordinary
// launch)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
// test-only fault injection (SBR_FAULT=alloc|timeout)
enum { kFaultNone = 0, kFaultAlloc = 1, kFaultTimeout = 2 };
int fault_mode();
// adds n to the launch count (kernel nodes of a CUDA graph launch; negative to
// take back launches that were only captured)
void note_launches(long long n);
// enqueue a device-side store of a value (no host buffer outlives the call)
sbr_status set_u64(unsigned long long* dst, unsigned long long v, cudaStream_t s);

// ---------------------------------------------------------------- icosahedron
struct Ico {
    double v[12][3];
    int8_t e[30][2];
    int8_t f[20][3];
};
Ico make_ico();

// ---------------------------------------------------------------- sort / scan
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
// keys/vals are sorted in place; tmp buffers are allocated on the stream.
sbr_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s);
// Exclusive prefix sum of n uint32 values, in place; *total (device, may be
// NULL) receives the sum.
sbr_status exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* total, cudaStream_t s);

// ---------------------------------------------------------------- BVH
// Node: 4 x float4 = child 0 box, child 1 box, refs. ref >= 0 internal node,
// ref < 0 leaf holding sorted primitive ~ref.
struct BvhNodes {
    float4* nodes = nullptr;   // [n_nodes * 4]
    int32_t* order = nullptr;  // [n] sorted position -> primitive index
    int32_t n_nodes = 0;       // internal nodes (>= 1 when n >= 1)
    float* d_root = nullptr;   // [6] root bounds on the device
};
// Build over n primitives given by boxes [n*6] (lo xyz, hi xyz) on the device.
// pad_rel: relative padding added to every child box (covers FP32 rounding).
// Subtrees of at most leaf_max (<= 16) primitives become one leaf; a leaf
// reference is ~(first | (count - 1) << 28).
// top_sah: rebuild the top of the tree with the surface-area heuristic
sbr_status build_lbvh(const float* prim_box, int64_t n, float pad_rel, int leaf_max, BvhNodes* out,
                      int32_t* d_depth, cudaStream_t s, bool top_sah = false);
constexpr int kTriLeaf = 2;  // triangles per BVH leaf at most (measured best of 1..6)
__host__ __device__ __forceinline__ int32_t leaf_first(int32_t ref) { return (~ref) & 0x0FFFFFFF; }
__host__ __device__ __forceinline__ int32_t leaf_count(int32_t ref) { return (int32_t)(((uint32_t)(~ref)) >> 28) + 1; }
void free_lbvh(BvhNodes* b, cudaStream_t s);

}  // namespace sbr

// ---------------------------------------------------------------- handles
struct sbr_bvh {
    int device = 0;
    int64_t T = 0;
    int32_t S = 0;
    sbr::BvhNodes tree;
    float4* tri_rot = nullptr;      // [3][T*3]: the faces below, vertex components rotated per
                                    //   block kz to (kz+1, kz+2, kz) mod 3 (FP32 hit tests)
    float4* tri_sorted = nullptr;   // [T*3] = block 2 of tri_rot: v0 (w = surface id bits),
                                    //   v1 (w = face id bits), v2
    float4* plane_sorted = nullptr; // [T*2] face plane as double-float, BVH order:
                                    //   (n_hi.xyz, c_hi), (n_lo.xyz, c_lo) with n.x = c
    float* tri = nullptr;           // [T*9] face-id order copy
    int32_t* surf = nullptr;        // [T]
    double* nrm = nullptr;          // [T*3] unit normal (FP64), face order
    int32_t* s_off = nullptr;       // [S+1] CSR of faces per surface
    int32_t* s_tri = nullptr;       // [T]   faces of each surface, ascending id
    int32_t* d_depth = nullptr;     // [1]
    cudaStream_t stream = nullptr;
};

struct TraceCountersDev {
    unsigned long long queue[SBR_KMAX + 2];  // rays entering bounce b
    unsigned long long work[SBR_KMAX + 2];   // work counters of the persistent grid
    unsigned long long candidates;
    unsigned long long keys;
    unsigned long long fp64_segments;
    unsigned long long fp64_tests;
    unsigned long long node_visits;  // instrumented traces only
    unsigned long long tri_tests;
    unsigned long long rx_visits;
    unsigned long long near_edge_hits;
    unsigned int status;
    unsigned int pad;
};

struct sbr_trace_result {
    int device = 0;
    sbr_trace_params params{};
    int64_t R = 0;                          // rays of the launch grid
    int64_t ray0 = 0, Rr = 0;               // traced id range [ray0, ray0 + Rr)
    int32_t n_rx = 0;
    double* rx = nullptr;                   // [n_rx*3] own copy
    double* d_alpha = nullptr;              // [1]
    int32_t table_log2 = 0;
    int32_t df_from = 0;                    // first bounce traced depth-first (K + 1: none)
    int32_t* seqf = nullptr;                // [K][Rr] face hit by each traced ray at each bounce
    uint32_t* ht_state = nullptr;           // [cap]
    uint32_t* ht_key = nullptr;             // [cap * kKeyWords]
    unsigned long long* ht_val = nullptr;   // [cap]
    TraceCountersDev* cnt = nullptr;
    cudaEvent_t ev[SBR_KMAX + 2] = {};     // bounce boundaries when timing is requested
    cudaStream_t stream = nullptr;
    // host copy of the final counters and alpha, taken by the path list's
    // first wait (the counters do not change once the trace launch has ended)
    mutable TraceCountersDev h_cnt{};
    mutable double h_alpha = 0.0;
    mutable bool h_valid = false;
};

struct sbr_path_list {
    int device = 0;
    int64_t P = 0, n_keys = 0, n_invalid = 0;
    int32_t n_rx = 0, K = 0, S = 0;
    double tx[3];
    double* rx_xyz = nullptr;   // [n_rx*3]
    int32_t* rx = nullptr;      // [P]
    int32_t* nb = nullptr;      // [P]
    int32_t* surf = nullptr;    // [P*8]
    int32_t* face = nullptr;    // [P*8]
    double* pts = nullptr;      // [P*8*3]
    double* L = nullptr;        // [P]
    double* aod = nullptr;      // [P*2]
    double* aoa = nullptr;      // [P*2]
    uint32_t* ray = nullptr;    // [P]
    float* dist = nullptr;      // [P]
    double* jones = nullptr;    // [P*kJones] polarimetric transfer data (gains)
    int32_t* rx_off = nullptr;  // [n_rx+1] paths of receiver r: [rx_off[r], rx_off[r+1])
    int32_t* h_rx_off = nullptr;  // host copy
    unsigned int* d_status = nullptr;  // device-side failures of later calls on this list
    cudaStream_t stream = nullptr;
};

namespace sbr {
// per-path polarimetric record for the gains kernel (FP64):
//   [0..1]   a1 (V): Tx theta-hat in the (s_1, p_in_1) basis      (LoS: [1, 0])
//   [2..3]   a1 (H): Tx phi-hat in the same basis                  (LoS: [1, 0])
//   [4..31]  M_k (k=1..7): 2x2 basis change (s_k, p_out_k) -> (s_k+1, p_in_k+1), row-major
//   [32..33] c (V): Rx theta-hat . (s_m, p_out_m)                  (LoS: [1, 0])
//   [34..35] c (H): Rx phi-hat . (s_m, p_out_m)                    (LoS: [1, 0])
//   [36..43] cos(theta_i) per reflection
constexpr int kJones = 48;

// launchers implemented in the .cu files
sbr_status launch_dirs(int32_t N, double* dirs, cudaStream_t s);
sbr_status launch_alpha(int32_t N, double* alpha, cudaStream_t s);
// the same alpha from one face of the lattice in double-float (the form a trace
// computes when it is given no alpha): ~1e-15 relative of the FP64 form
sbr_status launch_alpha_fast(int32_t N, double* alpha, cudaStream_t s);
sbr_status bvh_build(const float* tri, const int32_t* surf, int64_t T, int32_t S, sbr_bvh* b, cudaStream_t s,
                     bool sah_top);
sbr_status trace_run(const sbr_bvh* b, sbr_trace_result* tr, cudaStream_t s);
// the deduplicated records of a trace (sbr_trace_entries), synchronous
sbr_status trace_entries_run(const sbr_trace_result* tr, uint32_t* keys, unsigned long long* vals, int64_t cap,
                             int64_t* n_out, cudaStream_t s);
// a trace result built from records (sbr_trace_merge)
sbr_status trace_merge_run(sbr_trace_result* tr, const uint32_t* keys, const unsigned long long* vals, int64_t n,
                           cudaStream_t s);
sbr_status paths_run(const sbr_trace_result* tr, const sbr_bvh* b, sbr_path_list* pl,
                     cudaStream_t s);
sbr_status gains_run(const sbr_path_list* pl, const sbr_material* mats, int32_t S,
                     const double* freqs, int32_t F, const float* gamma, const float* disp,
                     int32_t pol, float2* g, cudaStream_t s);
sbr_status synth_simt_run(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                          const double* tx_elem, int32_t Nt, const double* rx_elem, int32_t Nr,
                          int32_t rx_index, bool fp64, float2* H, cudaStream_t s);
sbr_status synth_elements_run(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                              const double* tx_elem, int32_t Nt, bool fp64, float2* H, cudaStream_t s);
sbr_status synth_tc_run(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                        const double* tx_elem, int32_t Nt, const double* rx_elem, int32_t Nr,
                        int32_t rx_index, float2* H, bool f16, cudaStream_t s);
sbr_status pdp_run(const sbr_path_list* pl, const float2* g, int32_t F, int32_t f_index, double fc,
                   double bin_s, int32_t n_bins, float* pdp, double* stats, cudaStream_t s);
sbr_status surrogate_targets_run(const sbr_path_list* pl, const float2* g, int32_t F, int32_t n_taps,
                                double tap_s, double floor_db, float* out, cudaStream_t s);
sbr_status capacity_run(const float2* H, int32_t F, int32_t Nr, int32_t Nt, const double* snr_db,
                        int32_t n_snr, double* C, cudaStream_t s);
sbr_status capacity_noalloc_run(const float2* H, int32_t F, int32_t Nr, int32_t Nt,
                                const double* snr_db, int32_t n_snr, double* C, cudaStream_t s);
}  // namespace sbr

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__
namespace sbr {
struct d3 {
    double x, y, z;
};
__host__ __device__ __forceinline__ d3 mk3(double x, double y, double z) { return d3{x, y, z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return d3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return d3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 operator*(d3 a, double s) { return d3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
    return d3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(d3 a) { return sqrt(dot(a, a)); }
__device__ __forceinline__ d3 unit(d3 a) { return a * (1.0 / norm(a)); }
__device__ __forceinline__ d3 ld3(const double* p) { return d3{p[0], p[1], p[2]}; }
__device__ __forceinline__ void st3(double* p, d3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }
}  // namespace sbr
#endif
