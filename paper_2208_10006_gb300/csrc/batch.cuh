// Batched execution of many Tx-Rx jobs over several scenes: the device-side
// job records shared by the batched trace, path, gain and synthesis kernels.
#pragma once
#include "geodesic_df.cuh"
#include "sbr_internal.cuh"

namespace sbr {

constexpr int kBatchMaxJobsPerWave = 4096;   // job index packed in 12 bits of a ray record
constexpr int64_t kBatchMaxRaysPerJob = (int64_t)1 << 24;   // ray id packed in 24 bits

// One job (a Tx-Rx pair) as the batched kernels see it. Pointers are device
// memory owned by the batch (or by the caller, for the job's inputs and H).
struct BatchJobDev {
    // scene, BVH order (traversal)
    const float4* nodes;
    const float4* tris;
    const float4* plane;
    int64_t rot_stride;          // 3 T: float4s between the rotated copies of tris (tris is the last)
    // scene, face order (refinement) and materials (gains)
    const float* tri;
    const double* nrm;
    const int32_t* s_off;
    const int32_t* s_tri;
    const sbr_material* mats;
    int32_t S;
    // rays of the job
    int32_t R, K, wave_job;      // wave_job: index of the job within its wave
    GeoN geo;                    // subdivision of the launch grid (directions decoded per ray)
    int32_t* seq;                // [K][R] surface sequence (wave scratch)
    float tx_h[3], tx_l[3];      // Tx reference point, double-float
    float4 alpha;                // alpha hi, lo, alpha^2/3 hi, lo
    float4 rx_h, rx_l;           // Rx reference point, double-float (w unused)
    double tx[3], rx[3];         // the same points in FP64
    // synthesis inputs and output
    int32_t F, Nt, Nr, pol;
    const double* freqs;
    const float* gamma;
    const float* disp;
    const double* tx_elem;
    const double* rx_elem;
    float2* H;                   // [F][Nr][Nt]
    // per-job storage in the batch (capacity path_cap paths)
    int64_t path_base;           // first path slot of the job
    int64_t g_base;              // first gain, path-major [path_cap][F]
    // synthesis operands (wave scratch), rows of ps = the path capacity rounded up to 8
    int64_t w_base;              // first reflected-path weight, frequency-major [F][ps]
    int64_t wl_base;             // first LoS weight and FP16 scale, [F] each
    int64_t dt_base, dr_base, dl_base;   // element delays, [Nt][ps], [Nr][ps], [Nr][Nt]
};

// Path records of the batch, SoA over path slots (job j owns slots
// [path_base, path_base + path_cap)).
struct BatchPathsDev {
    int32_t* nb;
    int32_t* surf;      // [slot][kKmax]
    int32_t* face;      // [slot][kKmax]
    double* pts;        // [slot][kKmax][3]
    double* L;
    double* aod;        // [slot][2]
    double* aoa;
    uint32_t* ray;
    float* dist;
    double* jones;      // [slot][kJones]
};

// Device buffers of one wave of the batched trace.
struct BatchTraceWave {
    IcoLattice ico;              // launch grid decoded per ray
    const BatchJobDev* jobs;     // the wave's jobs
    const int64_t* ray_off;      // [n_jobs + 1] first global ray of each job in the wave
    int32_t n_jobs;
    int32_t Kmax;
    int64_t R_total;
    void* q0;                    // ray queues, 64 B records, capacity R_total each (breadth first)
    void* q1;
    bool depth_first;            // one launch, each ray carried through its bounces (no queues)
    uint32_t* ht_state;
    uint32_t* ht_key;
    unsigned long long* ht_val;
    uint32_t ht_mask;
    TraceCountersDev* cnt;
};

// launches the K_max + 1 bounces of one wave on s (no allocation, no host
// synchronisation: capturable in a CUDA graph)
sbr_status batch_trace_wave(const BatchTraceWave& w, int blocks_per_sm, cudaStream_t s);
int batch_trace_kernels(int Kmax);   // launches batch_trace_wave makes
int batch_trace_occupancy(bool depth_first);   // resident blocks per SM of the batched trace kernel

}  // namespace sbr

namespace sbr {
// batched tensor-core synthesis of one wave (synth_tc.cu)
struct BatchSynthWave {
    const BatchJobDev* jobs;
    const int64_t* item_off;     // [n_jobs + 1] for the wave's tile width
    int32_t n_jobs;
    int64_t items;
    const int32_t* np;           // [n_jobs] paths per job
    const int32_t* nb;           // reflections per path slot (batch path store)
    int32_t path_cap;            // row length of w, dt, dr: the path capacity rounded up to 8
    const float* dt;
    const float* dr;
    const float* dl;
    const float2* w;
    const float2* wl;
    const float* sc;
    unsigned int* status;
};
// tiles of one job for a tile width (64 receive elements x tile_n transmit elements per frequency)
inline int64_t batch_synth_items(int32_t F, int32_t Nr, int32_t Nt, int tile_n) {
    return (int64_t)F * ((Nr + 63) / 64) * ((Nt + tile_n - 1) / tile_n);
}
sbr_status batch_synth_prepare(bool f16, int tile_n);   // kernel attributes; call before capture
sbr_status batch_synth_tc(const BatchSynthWave& w, bool f16, int tile_n, cudaStream_t s);
}  // namespace sbr
