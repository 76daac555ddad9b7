/*
 * sbr.h - C ABI of the GB300 (sm_103a) SBR channel-modelling library.
 *
 * Implements the data-parallel hot path of "An SBR Based Ray Tracing Channel
 * Modeling Method for THz and Massive MIMO Communications" (arXiv
 * 2208.10006): geodesic ray launching (Sec. II-A.1), shoot-and-bounce tracing
 * with reception spheres (Sec. II-A.2, II-A.3), duplicate-path removal,
 * image-method refinement, path gains with Fresnel x Kirchhoff roughness and
 * atmospheric absorption (Eq. 1, 3, 6-10), near-field MIMO H(f) synthesis
 * (Eq. 11-14), PDP / delay spread / angles (Eq. 2, 4, 5) and capacity
 * (Eq. 15-17).
 *
 * Conventions (all entry points):
 *  - Plain C types only. Pointers marked "dev" are CUDA device pointers owned
 *    by the caller; "host" pointers are read before the call returns.
 *    Handles (sbr_bvh, sbr_trace_result, sbr_path_list) are owned by the
 *    library and released with their *_free function (NULL is accepted).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls enqueue work on it and return without waiting unless
 *    marked "synchronous".
 *  - Units: metres, hertz, siemens per metre; angles out in degrees.
 *  - Inputs are validated on the host before any launch; a failed check
 *    returns SBR_ERR_INVALID_ARG and launches nothing. No call traps or
 *    asserts on the device: device-side failures (a full dedup table, a
 *    traversal stack overflow, a bounded wait that ran out) are recorded in a
 *    status word and returned by the next synchronous call.
 *  - sbr_last_error() returns a thread-local message for the last failure.
 *  - Every call works on the current CUDA device; handles must be used on the
 *    device they were created on.
 */
#ifndef SBR_H
#define SBR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SBR_OK = 0,
    SBR_ERR_INVALID_ARG = 1,    /* bad pointer, size or parameter               */
    SBR_ERR_CUDA = 2,           /* a CUDA runtime call failed                   */
    SBR_ERR_CAPACITY = 3,       /* dedup table full: retry with larger table_log2 */
    SBR_ERR_STACK_OVERFLOW = 4, /* BVH deeper than the traversal stack          */
    SBR_ERR_TIMEOUT = 5,        /* a bounded device wait gave up                */
    SBR_ERR_NUMERIC = 6,        /* non-finite input or result                   */
    SBR_ERR_UNSUPPORTED = 7,    /* valid request the library cannot serve       */
    SBR_ERR_ALLOC = 8           /* device allocation failed                      */
} sbr_status;

#define SBR_KMAX 8          /* maximum reflections per path                      */
#define SBR_POL_V 0         /* theta-hat polarisation at both ends               */
#define SBR_POL_H 1         /* phi-hat polarisation at both ends                 */

/* precision of sbr_synthesize_H */
#define SBR_SYNTH_FP64 0    /* FP64 CUDA-core summation                          */
#define SBR_SYNTH_FP32 1    /* FP32 CUDA-core summation, FP64 delay phase        */
#define SBR_SYNTH_BF16X3 2  /* tcgen05 BF16 hi/lo split (3 products), FP32 TMEM  */
#define SBR_SYNTH_FP16X3 3  /* tcgen05 FP16 hi/lo split (3 products), weights scaled
                               per frequency by a power of two, FP32 TMEM          */

/* number of stats columns written by sbr_pdp_angles */
#define SBR_NSTATS 7

/* Thread-local description of the last failure on this thread ("" if none). */
const char* sbr_last_error(void);

/* Library version string. */
const char* sbr_version(void);

/* Number of CUDA kernels this library has launched in the calling process
 * (all devices, all threads); for accounting, e.g. launches per pipeline step. */
int64_t sbr_launch_count(void);

typedef struct sbr_bvh sbr_bvh;
typedef struct sbr_trace_result sbr_trace_result;
typedef struct sbr_path_list sbr_path_list;

/* Per-surface material: relative permittivity, conductivity (S/m) and the
 * Kirchhoff roughness standard deviation (m) of Eq. 7. */
typedef struct {
    double eps_r;
    double sigma_s_per_m;
    double rough_m;
} sbr_material;

/*
 * sbr_launch_dirs - geodesic launch directions (Sec. II-A.1, Fig. 1).
 * Class-I frequency-N subdivision of the icosahedron, projected to the unit
 * sphere; R = 10 N^2 + 2 directions in the order: 12 vertices, then the N-1
 * interior points of each of the 30 edges (sorted vertex pairs), then the
 * interior points of each of the 20 faces (sorted vertex triples, row i
 * outer). dirs: dev double [R*3] (x,y,z per ray). alpha: dev double [1] or
 * NULL; receives the largest angle (rad) between directions joined by a
 * sub-triangle edge, the ray spacing that sizes the reception sphere.
 * N in [1, 20000].
 */
sbr_status sbr_launch_dirs(int32_t N, double* dirs, double* alpha, void* stream);

/*
 * sbr_build_bvh - acceleration structure over the scene triangles (the paper
 * gives none; Sec. III-C only says the intersection search is parallelised).
 * tri_xyz: dev float [T*9], vertices v0,v1,v2 (x,y,z) per triangle, face id =
 * index, T < 2^28. surface_id: dev int32 [T] in [0, S): coplanar faces that form one
 * reflecting surface share an id. T may be 0 (an empty scene). The handle
 * keeps its own copies; the inputs may be freed once the stream has run.
 * *out receives the handle (library-owned; sbr_bvh_free).
 */
sbr_status sbr_build_bvh(const float* tri_xyz, const int32_t* surface_id, int64_t T, int32_t S,
                         sbr_bvh** out, void* stream);

/* flags of sbr_build_bvh_ex */
#define SBR_BVH_SAH_TOP 1   /* rebuild the top of the tree with the surface-area heuristic */

/*
 * sbr_build_bvh_ex - sbr_build_bvh with build options (same arguments,
 * ownership and errors; flags 0 gives the same tree). SBR_BVH_SAH_TOP
 * rebuilds the levels above the subtrees of at most max(8, T/400) triangles
 * (about 650 of them) with a binned surface-area-heuristic build: on the
 * 51,600-triangle urban scene 7% fewer node visits per segment for about
 * 0.45 ms more build time, so it pays for scenes traced many times (batches,
 * many transmitters), not for one trace per build. Unknown flags are rejected.
 */
sbr_status sbr_build_bvh_ex(const float* tri_xyz, const int32_t* surface_id, int64_t T, int32_t S,
                            uint32_t flags, sbr_bvh** out, void* stream);
void sbr_bvh_free(sbr_bvh* bvh);

typedef struct {
    int64_t T;
    int32_t S;
    int32_t n_nodes;   /* internal nodes */
    int32_t depth;     /* maximum leaf depth */
    int32_t reserved;
} sbr_bvh_info;

/* Synchronous: waits for the build and reports its shape. */
sbr_status sbr_bvh_query(const sbr_bvh* bvh, sbr_bvh_info* out);

/*
 * sbr_trace - shoot and bounce (Sec. II-A.2, II-A.3).
 * Rays start at tx (the Tx reference point) along the sbr_launch_dirs set.
 * Each segment finds the nearest face (smallest t > 0, ties to the lower
 * face id), ignoring every face of the surface reflected last. For bounce
 * b = 0..max_bounces the segment [0, t_hit] is tested against every
 * receiver: t* = (Rx - o).d, received when 0 <= t* <= t_hit and
 * |o + t* d - Rx| <= alpha (L + t*) / sqrt(3), L the unfolded length before
 * the segment. Then the ray reflects specularly, d' = d - 2 (d.n) n, until
 * max_bounces reflections or escape. Received (rx, surface sequence) keys
 * are deduplicated on the device, keeping the minimum distance (ties to the
 * lower ray id).
 * rx_xyz: dev double [n_rx*3] (copied; may be freed after the stream runs).
 * alpha: 0 = computed as in sbr_launch_dirs. table_log2: 0 = automatic.
 * max_bounces in [0, 8]; n_rx in [0, 2^20]; 10 N^2 + 2 < 2^32.
 * ray_begin, ray_end: trace only the launch directions with geodesic ids in
 * [ray_begin, ray_end) (ray_end = 0: up to R); rays are independent (Sec. I
 * traces them in parallel), so traces of disjoint ranges, e.g. one per GPU,
 * merged with sbr_trace_entries and sbr_trace_merge give the path list of
 * the whole grid. 0 <= ray_begin < end <= R.
 * depth_first_from: bounces before it run breadth first (one launch per
 * bounce over a compacted queue of live rays, the "width first" order of
 * Sec. I); from it on, each thread carries its ray through every remaining
 * bounce and then takes the next ray (one launch, no queue). 0 (the
 * default) traces everything depth first; max_bounces + 1 or more traces
 * everything breadth first. The results are the same; only the schedule
 * differs.
 */
typedef struct {
    double tx[3];
    const double* rx_xyz;
    int32_t n_rx;
    int32_t subdiv_N;
    int32_t max_bounces;
    int32_t table_log2;
    double alpha;
    uint32_t flags;
    int32_t depth_first_from;
    int64_t ray_begin;       /* traced geodesic ids [ray_begin, ray_end); ray_end 0 = R */
    int64_t ray_end;
} sbr_trace_params;

/* sbr_trace_params.flags */
#define SBR_TRACE_TIMING 1u        /* record CUDA events around each bounce launch (bounce_ms) */
#define SBR_TRACE_COUNT_VISITS 2u  /* instrumented kernel: count BVH node visits, triangle tests
                                      and near-edge closest hits */

typedef struct {
    int64_t rays;
    int64_t ray_bounces;        /* segments traced: a ray with k reflections adds k+1 */
    int64_t candidates;         /* receptions before dedup                          */
    int64_t keys;               /* distinct (rx, surface sequence) keys             */
    int64_t fp64_segments;      /* segments re-traversed entirely in FP64           */
    int64_t fp64_tests;         /* faces re-decided by an exact FP64 test           */
    int64_t node_visits;        /* BVH nodes fetched (SBR_TRACE_COUNT_VISITS only)  */
    int64_t tri_tests;          /* triangle tests (SBR_TRACE_COUNT_VISITS only)     */
    int64_t rx_visits;          /* receiver-BVH nodes fetched (SBR_TRACE_COUNT_VISITS only) */
    int64_t near_edge_hits;     /* closest hits whose smallest FP64 barycentric is <= 1e-6
                                   (SBR_TRACE_COUNT_VISITS only): the GPU's own count of the
                                   edge-ambiguous hits the parity rule exempts */
    int64_t queue[SBR_KMAX + 2];/* rays alive at the start of each bounce           */
    double alpha;
    int32_t status;             /* sbr_status of the device-side checks             */
    int32_t table_log2;
    float bounce_ms[SBR_KMAX + 1]; /* device time of each bounce launch (SBR_TRACE_TIMING) */
    int32_t reserved;
} sbr_trace_counters;

sbr_status sbr_trace(const sbr_bvh* bvh, const sbr_trace_params* params, sbr_trace_result** out,
                     void* stream);
/* Synchronous: waits for the trace and returns its counters and status. After
 * sbr_paths on the same result the final counters are already on the host
 * (read by that call's first wait, when the trace had ended) and are returned
 * without a device round trip. */
sbr_status sbr_trace_stats(const sbr_trace_result* tr, sbr_trace_counters* out);
void sbr_trace_free(sbr_trace_result* tr);

/*
 * sbr_trace_entries - the deduplicated receptions of a trace as plain records
 * (Sec. II-A.2 "pick out effective paths"): one per (receiver, surface
 * sequence), with the minimum reception distance and, on a tie, the lowest ray
 * id. This is what the traces of disjoint ray ranges exchange before their
 * paths are refined. Synchronous (waits for the trace). keys: dev uint32
 * [cap*10] per record (receiver, reflections, 8 surface ids padded with
 * 0xffffffff); vals: dev uint64 [cap] (bits of the FP32 distance << 32 | ray
 * id). *n_out receives the record count; if it exceeds cap nothing is written
 * and SBR_ERR_CAPACITY is returned. The record order is unspecified. A trace
 * that failed on the device returns its status.
 */
sbr_status sbr_trace_entries(const sbr_trace_result* tr, uint32_t* keys, uint64_t* vals, int64_t cap,
                             int64_t* n_out, void* stream);
/*
 * sbr_trace_merge - a trace result holding the union of records (from
 * sbr_trace_entries of any number of traces of the same scene, launch grid,
 * receivers and max_bounces, in any order): per key the minimum value, the rule
 * of the trace's own deduplication, which is commutative and associative, so
 * sbr_paths on the merged result gives the path list of one trace over the
 * union of the ray ranges, bit for bit (its refinement takes no per-ray hints).
 * params: as given to those traces (ray range, depth_first_from and flags
 * ignored; table_log2 0 = sized from n). keys, vals: dev, layouts of
 * sbr_trace_entries, n records (may be 0). sbr_trace_stats of the result
 * reports the key count and zero ray counters. Asynchronous. A table too small
 * for the keys reports SBR_ERR_CAPACITY through sbr_trace_stats / sbr_paths.
 */
sbr_status sbr_trace_merge(const sbr_trace_params* params, const uint32_t* keys, const uint64_t* vals, int64_t n,
                           sbr_trace_result** out, void* stream);

/*
 * sbr_paths - effective paths (Sec. II-A.2 "pick out effective paths",
 * image method of Sec. I). Synchronous. The dedup table is compacted and
 * sorted by (rx, n_bounce, surface sequence); each key is refined in FP64:
 * the Tx is mirrored through the surface planes in order, the path is
 * back-traced from the Rx, and it is kept when every intersection parameter
 * lies in (0, 1) and every point lies inside one of its surface's triangles
 * (barycentric tolerance 1e-9). The reported face of each point is the
 * lowest-id such triangle; L = |image - Rx|. Invalid keys are dropped and
 * counted. *n_paths_out receives the number of valid paths P.
 */
sbr_status sbr_paths(const sbr_trace_result* tr, const sbr_bvh* bvh, sbr_path_list** out,
                     int64_t* n_paths_out, void* stream);

typedef struct {
    int64_t n_paths;
    int64_t n_keys;       /* before refinement */
    int64_t n_invalid;    /* dropped by refinement */
    int32_t n_rx;
    int32_t max_bounces;
    int32_t status;       /* device-side failures of calls on this list so far */
    int32_t reserved;
} sbr_path_info;

/* Synchronous: waits for the list's stream and also reports (in status and
 * as the return value) any device-side failure recorded by earlier
 * asynchronous calls on this list, e.g. a bounded wait that gave up in
 * sbr_synthesize_H. */
sbr_status sbr_path_query(const sbr_path_list* pl, sbr_path_info* out);

/*
 * sbr_path_export - copy the path list into caller buffers (device memory, or
 * host memory: pinned for the copy to stay asynchronous; any may be NULL). Layouts for P paths: rx, n_bounce int32 [P]; surf_seq, face_seq
 * int32 [P*8] (-1 padded); pts double [P*8*3] interaction points; length
 * double [P] (m); aod, aoa double [P*2] (azimuth, elevation from the
 * horizontal, degrees; AoD towards the first interaction point, AoA towards
 * the last); ray_id uint32 [P] (kept candidate); dist float [P] (its
 * distance to the Rx at reception).
 */
sbr_status sbr_path_export(const sbr_path_list* pl, int32_t* rx, int32_t* n_bounce,
                           int32_t* surf_seq, int32_t* face_seq, double* pts, double* length,
                           double* aod, double* aoa, uint32_t* ray_id, float* dist, void* stream);
void sbr_path_list_free(sbr_path_list* pl);

/*
 * sbr_path_gains - complex path gain g_n(f) (Eq. 1, 3, 6-10).
 * Per reflection: lossy Fresnel TE/TM with eta = eps_r - j sigma/(2 pi f eps0)
 * times the roughness factor rho = exp(-g/2), g = (4 pi sigma_h cos(theta_i) f / c)^2
 * (Eq. 6-8), tracked polarimetrically (E <- rho [G_TE (E.s) s + G_TM (E.p_in) p_out]);
 * free-space amplitude c / (4 pi f L) (Eq. 3 with unit power and beta = 1),
 * absorption 10^(-gamma(f) L / 20000) (Eq. 9, gamma in dB/km) and dispersion
 * phase -phi(f) (pi/180) L / 1000 (Eq. 10, phi in deg/km); projected on the
 * Rx polarisation. The delay phasor exp(-j 2 pi f L / c) is not included.
 * mats: dev sbr_material [S] indexed by surface id. freqs_hz: dev double [F].
 * gamma_db_km, disp_deg_km: dev float [F] or NULL (zero). pol: SBR_POL_V/H.
 * gains: dev complex64 [P*F] (re, im interleaved), path-major; may be NULL when P = 0.
 */
sbr_status sbr_path_gains(const sbr_path_list* pl, const sbr_material* mats, int32_t S,
                          const double* freqs_hz, int32_t F, const float* gamma_db_km,
                          const float* disp_deg_km, int32_t pol, void* gains, void* stream);

/*
 * sbr_synthesize_H - MIMO channel matrix per frequency (Eq. 11-14) with the
 * near-field spherical wavefront (Sec. I). For the paths of receiver
 * rx_index, with first/last interaction points P1/Pm:
 *   H[f,q,p] = sum_n g_n(f) exp(-j 2 pi f (L_n + dt_pn + dr_qn) / c),
 *   dt_pn = |T_p - P1| - |T_0 - P1|,  dr_qn = |R_q - Pm| - |R_0 - Pm|,
 * T_0 = the trace's tx, R_0 = rx_xyz[rx_index]; a LoS path uses the exact
 * |T_p - R_q| in its phase. gains: dev complex64 [P*F] from sbr_path_gains (NULL when P = 0).
 * tx_elem: dev double [Nt*3]; rx_elem: dev double [Nr*3].
 * precision: SBR_SYNTH_FP64 / FP32 (CUDA cores) or SBR_SYNTH_BF16X3 /
 * SBR_SYNTH_FP16X3 (tcgen05 tensor cores, U diag(w) V^T contraction, FP32
 * accumulation; FP16X3 keeps ~2^-22 of each operand where BF16X3 keeps ~2^-16).
 * H: dev complex64 [F*Nr*Nt], element (f, q, p) at (f*Nr + q)*Nt + p.
 */
sbr_status sbr_synthesize_H(const sbr_path_list* pl, const void* gains, const double* freqs_hz,
                            int32_t F, const double* tx_elem, int32_t Nt, const double* rx_elem,
                            int32_t Nr, int32_t rx_index, int32_t precision, void* H, void* stream);

/*
 * sbr_synthesize_H_elements - MIMO channel matrix with per-element reception
 * (Sec. I near field, Eq. 13-14; the spatial non-stationarity of Fig. 11).
 * Each receive element is a receiver of the trace (rx_xyz of the path list,
 * Nr = n_rx), so element q sees its own path set; its row sums those paths:
 *   H[f,q,p] = sum_{n: rx_n = q} g_n(f) exp(-j 2 pi f len_np / c),
 *   len_np = |T_p - R_q| for the LoS path, L_n + |T_p - P1| - |T_0 - P1|
 *   otherwise (P1 the first interaction point, T_0 the trace's tx).
 * Unlike sbr_synthesize_H no Rx-side correction is applied: the element is
 * the traced point. gains: dev complex64 [P*F] (NULL when P = 0);
 * freqs_hz: dev double [F]; tx_elem: dev double [Nt*3].
 * precision: SBR_SYNTH_FP64 or SBR_SYNTH_FP32 (summation type; element
 * delays and the reduced phase f L_n / c are always FP64).
 * H: dev complex64 [F*n_rx*Nt], element (f, q, p) at (f*n_rx + q)*Nt + p.
 * F, n_rx <= 65535. Device scratch: P*(Nt+F) doubles (plus the FP32 copies).
 */
sbr_status sbr_synthesize_H_elements(const sbr_path_list* pl, const void* gains, const double* freqs_hz,
                                     int32_t F, const double* tx_elem, int32_t Nt, int32_t precision,
                                     void* H, void* stream);

/*
 * sbr_pdp_angles - PDP and channel statistics per receiver (Eq. 2, 4, 5).
 * Uses column f_index of gains (F columns) at frequency fc_hz. PDP: absolute
 * delay tau = L / c in bins [k, k+1) * bin_s, tap = sum |g|^2 in dB (empty
 * bins -inf). stats per receiver: PL_coh = -10 log10 |sum g exp(-j 2 pi fc tau)|^2,
 * PL_inc = -10 log10 sum |g|^2, tau_rms (Eq. 5, s), power-weighted mean AoD
 * azimuth/elevation and AoA azimuth/elevation (deg). A receiver without
 * paths gets +inf path loss and NaN for the rest.
 * pdp_db: float [n_rx*n_bins]; stats: double [n_rx*SBR_NSTATS]; each in device
 * memory or in pinned host memory (cudaHostAlloc / cudaMallocHost, which
 * unified addressing makes device-accessible): the kernel writes the results
 * in place, complete when the stream has passed the call.
 */
sbr_status sbr_pdp_angles(const sbr_path_list* pl, const void* gains, int32_t F, int32_t f_index,
                          double fc_hz, double bin_s, int32_t n_bins, float* pdp_db,
                          double* stats, void* stream);

/*
 * sbr_capacity - MIMO capacity (Eq. 15-17). Eq. 16's factor Q = sum |h|^2 is
 * read as a Frobenius normalisation: W_f = (Nr Nt / Qbar) H_f H_f^H
 * (H_f^H H_f when Nt < Nr), Qbar = mean over f of ||H_f||_F^2; SNR linear
 * 10^(dB/10); C = mean_f log2 det(I + SNR/Nt W_f) by an FP64 Cholesky.
 * H: dev complex64 [F*Nr*Nt]; snr_db: host double [n_snr], 1 <= n_snr <= 32
 * (read before the call returns); C: dev double [n_snr] (bit/s/Hz).
 * min(Nr, Nt) <= 64 (the n x n Cholesky of one frequency is held in shared
 * memory); larger arrays return SBR_ERR_INVALID_ARG. Asynchronous: returns
 * once the work is enqueued on `stream`.
 */
sbr_status sbr_capacity(const void* H, int32_t F, int32_t Nr, int32_t Nt, const double* snr_db,
                        int32_t n_snr, double* C, void* stream);

/*
 * sbr_capacity_noalloc - sbr_capacity for callers that cannot allocate device
 * memory while they run (a host framework that owns the whole device memory
 * pool and forbids libraries from calling cudaMalloc, or a real-time loop held
 * to a fixed footprint after start-up). The paper has no counterpart: this is
 * an allocation policy, not a step of the method. Same result as sbr_capacity,
 * same arguments and layouts; it calls no cudaMalloc, cudaFree or allocating
 * routine. Its scratch is a fixed array inside the library of about 1.1 MB
 * that every GPU which loads the library holds until the process exits; hence
 * F <= 4096 and n_snr <= 32, larger requests return SBR_ERR_INVALID_ARG (use
 * sbr_capacity). The first call on a device looks up that array's address on
 * the device: make that first call before any stream capture. The address is
 * kept for the life of the process; after cudaDeviceReset the library's
 * module is loaded again and the kept address is stale, so do not call this
 * entry point after a device reset. All calls share
 * the array, so calls whose work overlaps on the GPU (e.g. on two streams at
 * once) race; serialise them. Every scratch value it reads is first written by
 * the same call. Asynchronous: returns once the work is enqueued on `stream`.
 */
sbr_status sbr_capacity_noalloc(const void* H, int32_t F, int32_t Nr, int32_t Nt, const double* snr_db,
                                int32_t n_snr, double* C, void* stream);

/* ------------------------------------------------------------------------
 * Batched execution: many Tx-Rx jobs (each one Tx reference point, one Rx
 * reference point, its own ray count, reflection depth, frequency grid and
 * arrays) over several scenes, run as one CUDA-graph launch. Per job the
 * result is that of sbr_trace + sbr_paths + sbr_path_gains +
 * sbr_synthesize_H on the same inputs (the same arithmetic in batched
 * kernels): Sec. II-A ray launching, tracing, reception and effective paths,
 * Eq. 1, 3, 6-10 gains and Eq. 13-14 synthesis, per job. Jobs are grouped
 * into waves whose rays fit the ray-queue capacity; each wave runs the
 * bounces as persistent launches over all of its jobs' rays, then the path,
 * gain and tensor-core synthesis kernels over all of its jobs.
 */
typedef struct sbr_batch sbr_batch;

typedef struct {
    int32_t scene;            /* index into the scenes given to sbr_batch_create           */
    int32_t subdiv_N;         /* rays R = 10 N^2 + 2, 1 <= N <= 1295 (R < 2^24)             */
    int32_t max_bounces;      /* K, 0..8                                                   */
    int32_t pol;              /* SBR_POL_V or SBR_POL_H, both ends                         */
    double tx[3];             /* Tx reference point (m)                                    */
    double rx[3];             /* Rx reference point (m)                                    */
    double alpha;             /* reception-sphere angle (rad); 0 = the launch grid's own   */
    int32_t F;                /* frequencies                                               */
    int32_t Nt;               /* transmit elements                                         */
    int32_t Nr;               /* receive elements                                          */
    int32_t reserved;
    const double* freqs_hz;   /* dev [F]                                                   */
    const float* gamma_db_km; /* dev [F] or NULL (Eq. 9)                                   */
    const float* disp_deg_km; /* dev [F] or NULL (Eq. 10)                                  */
    const double* tx_elem;    /* dev [Nt*3] element positions                              */
    const double* rx_elem;    /* dev [Nr*3]                                                */
    void* H;                  /* dev complex64 [F*Nr*Nt], written by sbr_batch_run          */
} sbr_batch_job;

typedef struct {
    int64_t wave_rays;        /* ray-queue capacity of a wave (rays); 0 = 2^26               */
    int32_t path_cap;         /* keys and paths kept per job; 0 = 512                       */
    int32_t table_log2;       /* dedup table slots per wave; 0 = from jobs per wave x path_cap */
    int32_t tile_n;           /* tensor-core tile width: 64, 128 or 256; 0 = 128             */
    int32_t trace_blocks_per_sm; /* persistent bounce grid; 0 = occupancy limit              */
    int32_t precision;        /* SBR_SYNTH_FP16X3 (0 = this) or SBR_SYNTH_BF16X3             */
    int32_t use_graph;        /* 1 (default when the config pointer is NULL): capture the   */
                              /* whole batch into one CUDA graph; 0: plain stream launches  */
    int32_t breadth_first;    /* 0 (default): each ray traced depth first through all its   */
                              /* bounces in one launch per wave; 1: one launch per bounce   */
                              /* over compacted ray queues                                  */
    int32_t reserved;
} sbr_batch_config;

typedef struct {
    int32_t n_jobs;
    int32_t n_waves;
    int32_t graph_kernels;    /* kernel nodes of one sbr_batch_run                          */
    int32_t status;           /* worst sbr_status over the jobs of the last run             */
    int32_t max_keys;         /* largest dedup key count of a job in the last run            */
    int32_t reserved;
    int64_t rays;             /* rays of all jobs                                           */
    int64_t ray_bounces;      /* segments traced in the last run                            */
    int64_t paths;            /* paths kept over all jobs in the last run                   */
    sbr_batch_config config;  /* the configuration in force (defaults resolved)             */
} sbr_batch_info;

/*
 * sbr_batch_create - validate the jobs, group them into waves, compute the
 * reception-sphere angle alpha of every distinct N (launch directions are
 * decoded from the ray id inside the trace, no table is built), and allocate
 * every buffer of the batch (no allocation happens in sbr_batch_run).
 * scenes: n_scenes BVH handles; mats[s]: dev array of scenes[s]'s surfaces
 * (at least its S entries). jobs: host array of n_jobs (copied). cfg may be
 * NULL (defaults). The scene handles and the jobs' device arrays must outlive
 * the batch. Synchronous. Errors: SBR_ERR_INVALID_ARG (a job or config field
 * out of range; nothing allocated), SBR_ERR_ALLOC.
 */
sbr_status sbr_batch_create(const sbr_bvh* const* scenes, const sbr_material* const* mats,
                            int32_t n_scenes, const sbr_batch_job* jobs, int32_t n_jobs,
                            const sbr_batch_config* cfg, sbr_batch** out, void* stream);
/*
 * sbr_batch_run - run every job; writes each job's H. With use_graph the
 * first call captures the batch into a CUDA graph on a stream of its own and
 * every call launches that graph on `stream`. Asynchronous; per-job failures
 * (a full dedup table or path store: SBR_ERR_CAPACITY, a bounded wait that
 * gave up: SBR_ERR_TIMEOUT) are reported by sbr_batch_query.
 */
sbr_status sbr_batch_run(sbr_batch* b, void* stream);
/*
 * sbr_batch_query - synchronous: per job the number of paths (n_paths, host
 * int32 [n_jobs], may be NULL) and its sbr_status (status, host int32
 * [n_jobs], may be NULL) of the last run, and the batch summary (info, may be
 * NULL). Returns the worst job status.
 */
sbr_status sbr_batch_query(const sbr_batch* b, int32_t* n_paths, int32_t* status, sbr_batch_info* info);
/*
 * sbr_batch_export - copy the first n paths of one job (n <= its n_paths) in
 * the layouts of sbr_path_export (receiver index implied: 0) and, if gains is
 * not NULL, its complex64 gains [n*F]. Device pointers may be NULL to skip a
 * field. Asynchronous on `stream`.
 */
sbr_status sbr_batch_export(const sbr_batch* b, int32_t job, int32_t n, int32_t* n_bounce,
                            int32_t* surf_seq, int32_t* face_seq, double* pts, double* length,
                            double* aod, double* aoa, uint32_t* ray_id, float* dist, void* gains,
                            void* stream);
void sbr_batch_free(sbr_batch* b);

/*
 * sbr_batch_tune - autotuner: for the given jobs (typically a sample of a
 * larger batch) time each candidate of tile_n x trace_blocks_per_sm x
 * wave_rays (its own batches, two warm runs and the median of three timed
 * ones), size path_cap to the largest path count seen (x 1.5, a power of two,
 * at least 64) and return the fastest configuration in *cfg (fields left
 * non-zero by the caller are kept fixed) and its time per run in *ms.
 * Synchronous.
 */
sbr_status sbr_batch_tune(const sbr_bvh* const* scenes, const sbr_material* const* mats,
                          int32_t n_scenes, const sbr_batch_job* jobs, int32_t n_jobs,
                          sbr_batch_config* cfg, double* ms, void* stream);

/* ------------------------------------------------------------------------
 * Learned surrogate. The paper has no counterpart: a query-time stand-in for
 * the method's per-receiver outputs (path loss, RMS delay spread and PDP of
 * Eq. 2, 4, 5), learned from them, with full SBR as the fallback and arbiter.
 */

/*
 * sbr_surrogate_targets - per receiver r and frequency f of a path list and
 * its gains (sbr_path_gains, [P*F]): out[(r*F + f)*(2 + n_taps) + k] =
 *   k = 0: incoherent path loss -10 log10 sum_n |g_n(f)|^2 (dB, Eq. 4 power sum)
 *   k = 1: RMS delay spread of Eq. 5 with P_n = |g_n(f)|^2, tau_n = L_n / c (s)
 *   k = 2 + i: PDP tap i, 10 log10 of the power with tau_n - tau_min in
 *              [i tap_s, (i + 1) tap_s) over the total (dB), floor_db when
 *              below it or empty.
 * A receiver without paths gets NaN everywhere. FP64 arithmetic, FP32 out.
 * n_taps in [1, 32]. Asynchronous.
 */
sbr_status sbr_surrogate_targets(const sbr_path_list* pl, const void* gains, int32_t F, int32_t n_taps,
                                 double tap_s, double floor_db, float* out, void* stream);

typedef struct sbr_mlp sbr_mlp;

typedef struct {
    int32_t n_out;          /* outputs used, <= 128                                         */
    int32_t width;          /* hidden width: 128 or 256                                     */
    int32_t depth;          /* hidden layers, 1..8                                          */
    int32_t max_batch;      /* rows per call, <= 2^22                                       */
    uint64_t seed;          /* initial weights (He-uniform from splitmix64)                 */
    float x_lo[4];          /* input box of (x, y, z, f), mapped to [0, 1] for the features */
    float x_hi[4];
    float lr, beta1, beta2, eps;   /* Adam                                                */
    int32_t err_channel;    /* output that learns |output err_of - its target|, or -1       */
    int32_t err_of;         /* (stop-gradient on output err_of), or -1                      */
    float feat_log2_max;    /* highest feature frequency pi 2^feat_log2_max (0 = 9)         */
    int32_t reserved;
} sbr_mlp_config;

/*
 * sbr_mlp_create - the MLP: 128 Fourier features of (x, y, z, f) (coordinate
 * c, octave k = 0..15: sin and cos of pi 2^(k m / 15) u_c, u = (x - x_lo) /
 * (x_hi - x_lo), m = feat_log2_max) -> depth ReLU layers of `width` -> 128 linear outputs, the
 * first n_out used. BF16 operands on the tcgen05 tensor cores, FP32
 * accumulation and FP32 master weights. loss_w: host [n_out] weights of the
 * squared errors (NULL: all 1); y_shift, y_scale: host [n_out] target
 * normalisation, the network learning (y - shift) / scale and predicting in
 * target units (NULL: 0 and 1). Synchronous.
 */
sbr_status sbr_mlp_create(const sbr_mlp_config* cfg, const float* loss_w, const float* y_shift,
                          const float* y_scale, sbr_mlp** out, void* stream);
/*
 * sbr_mlp_train_step - one Adam step on a batch: x dev [B*4], y dev [B*n_out]
 * targets (NaN = no target). Loss (1/B) sum w_o (p - y')^2 over finite targets
 * y' = (y - shift) / scale, plus, for the error head, (1/B) sum w_e
 * (p_e - |p_c - y'_c|)^2 (the head predicts in the normalised units of c,
 * times scale_e + shift_e when predicted). loss: dev
 * float accumulated with atomicAdd (zero it first), or NULL. Asynchronous.
 */
sbr_status sbr_mlp_train_step(sbr_mlp* m, const float* x, const float* y, int32_t B, float* loss, void* stream);
/*
 * sbr_mlp_predict - y dev [B*n_out] = outputs for x dev [B*4], in one fused
 * launch (every layer of 128 rows per CTA with the activations kept in shared
 * memory). sbr_mlp_predict_layered: the same outputs through the training
 * path's per-layer GEMMs (activations through device memory), for checking.
 * Asynchronous.
 */
sbr_status sbr_mlp_predict(const sbr_mlp* m, const float* x, int32_t B, float* y, void* stream);
sbr_status sbr_mlp_predict_layered(const sbr_mlp* m, const float* x, int32_t B, float* y, void* stream);
/* number of FP32 parameters (per layer: W [n_out][n_in] row-major, then b) */
int64_t sbr_mlp_param_count(const sbr_mlp* m);
/*
 * sbr_mlp_params - mode 0: copy the FP32 parameters to params (dev); 1: load
 * them from params (and refresh the BF16 copies); 2: copy the gradients of
 * the last training step. Layout of sbr_mlp_param_count. Asynchronous.
 */
sbr_status sbr_mlp_params(sbr_mlp* m, float* params, int32_t mode, void* stream);
/* learning rate of the following steps (a schedule is the caller's) */
sbr_status sbr_mlp_set_lr(sbr_mlp* m, float lr);
/* synchronous: SBR_ERR_TIMEOUT if a bounded tensor-core wait gave up */
sbr_status sbr_mlp_status(const sbr_mlp* m);
void sbr_mlp_free(sbr_mlp* m);

#ifdef __cplusplus
}
#endif
#endif /* SBR_H */
