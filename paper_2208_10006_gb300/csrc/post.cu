// Channel statistics (Eq. 2, 4, 5; the Table I quantities) and MIMO capacity
// (Eq. 15-17).
//
// PDP / stats: one block per receiver. tau = L / c, bin floor(tau / bin_s),
// tap = sum |g|^2 (FP64 accumulation), PL_coh from the coherent sum with the
// FP64-reduced delay phase, tau_rms from the power-weighted moments (Eq. 5),
// power-weighted mean AoD/AoA.
//
// Capacity: Eq. 16 multiplies W by Q = sum |h|^2, which read literally drives
// C to zero at realistic path loss; the reading used is the Frobenius
// normalisation W_f = (Nr Nt / Qbar) H_f H_f^H (H_f^H H_f when Nt < Nr),
// Qbar = mean_f ||H_f||_F^2. W_f is formed in FP32 on CUDA cores, then
// log2 det(I + SNR/Nt W_f) by an FP64 complex Cholesky in shared memory, one
// block per frequency; the per-(f, SNR) log-determinants are averaged over f
// in a fixed order.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "sbr_internal.cuh"

namespace sbr {
namespace {

constexpr int kPdpThreads = 256;

__device__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

__global__ void __launch_bounds__(kPdpThreads)
k_pdp(const int32_t* __restrict__ rx_off, const double* __restrict__ L, const double* __restrict__ aod,
      const double* __restrict__ aoa, const float2* __restrict__ g, int32_t F, int32_t f_index,
      double fc, double bin_s, int32_t n_bins, float* __restrict__ pdp, double* __restrict__ stats) {
    ::sbr::pdl_wait();
    extern __shared__ double acc[];  // [n_bins]
    const int r = blockIdx.x;
    const int32_t o0 = rx_off[r], o1 = rx_off[r + 1];
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) acc[k] = 0.0;
    __syncthreads();
    double sp = 0, st = 0, st2 = 0, cr = 0, ci = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    for (int32_t n = o0 + threadIdx.x; n < o1; n += blockDim.x) {
        float2 gg = g[(int64_t)n * F + f_index];
        double gr = gg.x, gi = gg.y;
        double pw = gr * gr + gi * gi;
        double tau = L[n] / kC0;
        double kb = floor(tau / bin_s);
        if (kb >= 0.0 && kb < (double)n_bins) atomicAdd(&acc[(int)kb], pw);
        sp += pw; st += pw * tau; st2 += pw * tau * tau;
        double cyc = fc * L[n] / kC0;
        double s, c;
        sincospi(-2.0 * (cyc - floor(cyc)), &s, &c);
        cr += gr * c - gi * s;
        ci += gr * s + gi * c;
        a1 += pw * aod[2 * n]; a2 += pw * aod[2 * n + 1];
        a3 += pw * aoa[2 * n]; a4 += pw * aoa[2 * n + 1];
    }
    {
        // the nine block sums at once, each in the order of block_sum (butterfly
        // within each warp, then the warps in order): two barriers instead of 27.
        // A receiver with at most 32 paths has them all in warp 0, whose sums
        // alone are added (the other warps' are exact zeros): the FP64 pipe,
        // this kernel's bound, then carries one warp's butterflies, not eight
        __shared__ double part[kPdpThreads / 32][9];
        __shared__ double tot[9];
        double v[9] = {sp, st, st2, cr, ci, a1, a2, a3, a4};
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const bool one_warp = o1 - o0 <= 32;
        if (!one_warp || warp == 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q)
                for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 9; ++q) part[warp][q] = v[q];
        }
        __syncthreads();
        if (threadIdx.x < 9) {
            double t = 0.0;
            const int nw = one_warp ? 1 : kPdpThreads / 32;
            for (int w = 0; w < nw; ++w) t += part[w][threadIdx.x];
            tot[threadIdx.x] = t;
        }
        __syncthreads();
        sp = tot[0]; st = tot[1]; st2 = tot[2]; cr = tot[3]; ci = tot[4];
        a1 = tot[5]; a2 = tot[6]; a3 = tot[7]; a4 = tot[8];
    }
    // a bin holds a sum of powers (>= 0): its bit pattern is positive exactly when
    // it is non-zero, which keeps the test of the (mostly empty) bins off the FP64 pipe
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) {
        const double v = acc[k];
        pdp[(int64_t)r * n_bins + k] = __double_as_longlong(v) > 0 ? (float)(10.0 * log10(v)) : -INFINITY;
    }
    if (threadIdx.x == 0) {
        double* o = stats + (int64_t)r * SBR_NSTATS;
        if (o1 == o0 || !(sp > 0.0)) {
            o[0] = INFINITY; o[1] = INFINITY;
            for (int k = 2; k < SBR_NSTATS; ++k) o[k] = NAN;
        } else {
            o[0] = -10.0 * log10(cr * cr + ci * ci);
            o[1] = -10.0 * log10(sp);
            double m1 = st / sp, m2 = st2 / sp, var = m2 - m1 * m1;
            o[2] = sqrt(var > 0.0 ? var : 0.0);
            o[3] = a1 / sp; o[4] = a2 / sp; o[5] = a3 / sp; o[6] = a4 / sp;
        }
    }
}

// ---------------------------------------------------------------- capacity
constexpr int kCapThreads = 256;
constexpr int kMaxSnr = 32;        // SNR values per capacity call

__global__ void k_frob(const float2* __restrict__ H, int64_t per_f, double* __restrict__ qf) {
    __shared__ double sh[33];
    const float2* h = H + (int64_t)blockIdx.x * per_f;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < per_f; i += blockDim.x) {
        float2 x = h[i];
        v += (double)x.x * x.x + (double)x.y * x.y;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) qf[blockIdx.x] = v;
}

__global__ void k_qbar(const double* __restrict__ qf, int32_t F, double* __restrict__ qbar) {
    double s = 0.0;
    for (int32_t f = 0; f < F; ++f) s += qf[f];
    *qbar = s / F;
}

// one block per frequency; n = min(Nr, Nt) <= 64
__global__ void __launch_bounds__(kCapThreads)
k_capacity(const float2* __restrict__ H, int32_t Nr, int32_t Nt, const double* __restrict__ snr_lin,
           int32_t n_snr, const double* __restrict__ qbar, double* __restrict__ ld) {
    extern __shared__ unsigned char smem[];
    const int n = Nr < Nt ? Nr : Nt;
    float2* W = reinterpret_cast<float2*>(smem);                           // [n*n]
    double2* A = reinterpret_cast<double2*>(smem + sizeof(float2) * ((n * n + 1) & ~1));  // [n*n]
    __shared__ double s_ld;
    __shared__ int s_bad;
    const int f = blockIdx.x;
    const float2* h = H + (int64_t)f * Nr * Nt;
    // W[a][b] = sum_p H[a][p] conj(H[b][p])  (Nt >= Nr)  or  sum_q conj(H[q][a]) H[q][b]
    // Blocked summation: FP32 partial sums over runs of kCapRun terms, added
    // into FP64 totals, so the rounding error of an entry grows with the run
    // length rather than with the array size (16,384 terms at a 128 x 128 UPA)
    constexpr int kCapRun = 32;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int a = e / n, b = e - a * n;
        double sre = 0.0, sim = 0.0;
        if (Nt >= Nr) {
            for (int p0 = 0; p0 < Nt; p0 += kCapRun) {
                const int p1 = min(Nt, p0 + kCapRun);
                float re = 0.f, im = 0.f;
                for (int p = p0; p < p1; ++p) {
                    float2 x = h[(int64_t)a * Nt + p], y = h[(int64_t)b * Nt + p];
                    re += x.x * y.x + x.y * y.y;
                    im += x.y * y.x - x.x * y.y;
                }
                sre += re;
                sim += im;
            }
        } else {
            for (int q0 = 0; q0 < Nr; q0 += kCapRun) {
                const int q1 = min(Nr, q0 + kCapRun);
                float re = 0.f, im = 0.f;
                for (int q = q0; q < q1; ++q) {
                    float2 x = h[(int64_t)q * Nt + a], y = h[(int64_t)q * Nt + b];
                    re += x.x * y.x + x.y * y.y;
                    im += x.x * y.y - x.y * y.x;
                }
                sre += re;
                sim += im;
            }
        }
        W[e] = make_float2((float)sre, (float)sim);
    }
    __syncthreads();
    const double scale = (double)Nr * Nt / *qbar;
    for (int si = 0; si < n_snr; ++si) {
        const double c = snr_lin[si] / Nt * scale;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int a = e / n, b = e - a * n;
            A[e] = make_double2((a == b ? 1.0 : 0.0) + c * W[e].x, c * W[e].y);
        }
        if (threadIdx.x == 0) { s_ld = 0.0; s_bad = 0; }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            if (threadIdx.x == 0) {
                double d = A[j * n + j].x;
                if (!(d > 0.0)) { s_bad = 1; d = 1.0; }
                double l = sqrt(d);
                A[j * n + j] = make_double2(l, 0.0);
                s_ld += 2.0 * log(l);
            }
            __syncthreads();
            const double inv = 1.0 / A[j * n + j].x;
            for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
                double2 v = A[i * n + j];
                A[i * n + j] = make_double2(v.x * inv, v.y * inv);
            }
            __syncthreads();
            const int m = n - j - 1;
            for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
                int i = j + 1 + e / m, k = j + 1 + e % m;
                if (k > i) continue;
                double2 lij = A[i * n + j], lkj = A[k * n + j];
                double2 v = A[i * n + k];
                // A[i][k] -= L[i][j] conj(L[k][j])
                v.x -= lij.x * lkj.x + lij.y * lkj.y;
                v.y -= lij.y * lkj.x - lij.x * lkj.y;
                A[i * n + k] = v;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) ld[(int64_t)f * n_snr + si] = s_bad ? NAN : s_ld;
        __syncthreads();
    }
}

__global__ void k_cap_reduce(const double* __restrict__ ld, int32_t F, int32_t n_snr,
                             double* __restrict__ C) {
    int si = threadIdx.x;
    if (si >= n_snr) return;
    double s = 0.0;
    for (int32_t f = 0; f < F; ++f) s += ld[(int64_t)f * n_snr + si];
    C[si] = s / F / log(2.0);
}

// linear SNR values of one capacity call, passed by value in the launch
struct SnrList {
    double lin[kMaxSnr];
};

__global__ void k_snr_store(const __grid_constant__ SnrList snr, int32_t n, double* __restrict__ out) {
    int i = threadIdx.x;
    if (i < n) out[i] = snr.lin[i];
}

// surrogate targets: one warp per (receiver, frequency); FP64 sums over the
// receiver's paths of P_n = |g_n(f)|^2, tau_n = L_n / c, relative to the first
// arrival for the delay spread and the taps
__global__ void k_surrogate_targets(const int32_t* __restrict__ rx_off, int32_t n_rx, const float2* __restrict__ g,
                                    const double* __restrict__ L, int32_t F, int32_t n_taps, double tap_s,
                                    double floor_db, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)n_rx * F) return;
    const int r = (int)(w / F), f = (int)(w - (int64_t)r * F);
    const int p0 = rx_off[r], p1 = rx_off[r + 1];
    const int stride = 2 + n_taps;
    float* o = out + w * stride;
    if (p1 == p0) {
        for (int k = lane; k < stride; k += 32) o[k] = NAN;
        return;
    }
    double tmin = INFINITY;
    for (int p = p0 + lane; p < p1; p += 32) tmin = fmin(tmin, L[p] / kC0);
    for (int s = 16; s; s >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, s));
    double sp = 0.0, st = 0.0, st2 = 0.0;
    double tap[32];
    for (int k = 0; k < 32; ++k) tap[k] = 0.0;
    for (int p = p0 + lane; p < p1; p += 32) {
        float2 gg = g[(int64_t)p * F + f];
        double pw = (double)gg.x * gg.x + (double)gg.y * gg.y;
        double t = L[p] / kC0 - tmin;
        sp += pw;
        st += pw * t;
        st2 += pw * t * t;
        double b = floor(t / tap_s);
        if (b >= 0.0 && b < n_taps) {
            int bi = (int)b;
            for (int k = 0; k < 32; ++k) tap[k] += k == bi ? pw : 0.0;
        }
    }
    for (int s = 16; s; s >>= 1) {
        sp += __shfl_xor_sync(0xffffffffu, sp, s);
        st += __shfl_xor_sync(0xffffffffu, st, s);
        st2 += __shfl_xor_sync(0xffffffffu, st2, s);
        for (int k = 0; k < 32; ++k) tap[k] += __shfl_xor_sync(0xffffffffu, tap[k], s);
    }
    if (lane != 0) return;
    o[0] = (float)(-10.0 * log10(sp));
    double mean = st / sp;
    o[1] = (float)sqrt(fmax(st2 / sp - mean * mean, 0.0));
    for (int k = 0; k < n_taps; ++k) {
        double db = tap[k] > 0.0 ? 10.0 * log10(tap[k] / sp) : floor_db;
        o[2 + k] = (float)fmax(db, floor_db);
    }
}

}  // namespace

sbr_status pdp_run(const sbr_path_list* pl, const float2* g, int32_t F, int32_t f_index, double fc,
                   double bin_s, int32_t n_bins, float* pdp, double* stats, cudaStream_t s) {
    if (pl->n_rx == 0) return SBR_OK;
    size_t smem = sizeof(double) * (size_t)n_bins;
    if (smem > 48 * 1024)
        SBR_TRY_CUDA(cudaFuncSetAttribute(k_pdp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_pdp, dim3(pl->n_rx), dim3(kPdpThreads), smem, s, pl->rx_off, pl->L, pl->aod, pl->aoa, g, F, f_index, fc,
                                               bin_s, n_bins, pdp, stats);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

size_t capacity_smem(int32_t Nr, int32_t Nt) {
    int n = std::min(Nr, Nt);
    return sizeof(float2) * (size_t)((n * n + 1) & ~1) + sizeof(double2) * (size_t)n * n;
}

sbr_status surrogate_targets_run(const sbr_path_list* pl, const float2* g, int32_t F, int32_t n_taps,
                                double tap_s, double floor_db, float* out, cudaStream_t s) {
    if (pl->n_rx == 0) return SBR_OK;
    int64_t threads = (int64_t)pl->n_rx * F * 32;
    ::sbr::note_launch(), k_surrogate_targets<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        pl->rx_off, pl->n_rx, g, pl->L, F, n_taps, tap_s, floor_db, out);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

sbr_status capacity_run(const float2* H, int32_t F, int32_t Nr, int32_t Nt, const double* snr_db,
                        int32_t n_snr, double* C, cudaStream_t s) {
    // the linear SNR list travels by value in the first launch, so the call
    // returns as soon as its work is enqueued (no host table has to outlive it)
    SnrList snr{};
    for (int i = 0; i < n_snr; ++i) snr.lin[i] = std::pow(10.0, snr_db[i] / 10.0);
    double *d_lin, *qf, *qbar, *ld;
    SBR_TRY(dalloc_n(&d_lin, n_snr, s));
    SBR_TRY(dalloc_n(&qf, F, s));
    SBR_TRY(dalloc_n(&qbar, 1, s));
    SBR_TRY(dalloc_n(&ld, (size_t)F * n_snr, s));
    ::sbr::note_launch(), k_snr_store<<<1, kMaxSnr, 0, s>>>(snr, n_snr, d_lin);
    ::sbr::note_launch(), k_frob<<<F, kCapThreads, 0, s>>>(H, (int64_t)Nr * Nt, qf);
    ::sbr::note_launch(), k_qbar<<<1, 1, 0, s>>>(qf, F, qbar);
    size_t smem = capacity_smem(Nr, Nt);
    SBR_TRY_CUDA(cudaFuncSetAttribute(k_capacity, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ::sbr::note_launch(), k_capacity<<<F, kCapThreads, smem, s>>>(H, Nr, Nt, d_lin, n_snr, qbar, ld);
    ::sbr::note_launch(), k_cap_reduce<<<1, 32, 0, s>>>(ld, F, n_snr, C);
    SBR_TRY_CUDA(cudaGetLastError());
    dfree(d_lin, s); dfree(qf, s); dfree(qbar, s); dfree(ld, s);
    return SBR_OK;
}


// ---------------------------------------------------------------- capacity without allocation
// Some callers cannot allocate device memory once they are running: a host
// framework that owns the whole device memory pool and forbids libraries from
// calling cudaMalloc, or a real-time simulation loop held to a fixed memory
// footprint after start-up. sbr_capacity_noalloc serves them: the same
// kernels as sbr_capacity, with every scratch buffer placed in the fixed
// array below, which each GPU that loads the library holds until the process
// exits (about 1.1 MB).
constexpr int kNoAllocMaxF = 4096;    // frequencies per call
constexpr int kNoAllocMaxSnr = kMaxSnr;  // SNR values per call

struct CapacityScratch {
    double qf[kNoAllocMaxF];                     // ||H_f||_F^2
    double qbar;                                 // mean over f
    double snr_lin[kNoAllocMaxSnr];              // 10^(dB/10)
    double ld[kNoAllocMaxF * kNoAllocMaxSnr];    // ln det per (f, SNR)
};
static __device__ __align__(256) CapacityScratch g_capacity_scratch;

namespace {

std::mutex g_scratch_mu;
CapacityScratch* g_scratch_ptr[256] = {};

// device address of the scratch array on the current device; looked up once
// per device (the first call on a device does it)
sbr_status capacity_scratch(CapacityScratch** out) {
    int dev = 0;
    SBR_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal %d out of range", dev);
        return SBR_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_capacity_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("cudaGetSymbolAddress(capacity scratch) failed: %s", cudaGetErrorString(e));
            return SBR_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<CapacityScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
    return SBR_OK;
}

}  // namespace

sbr_status capacity_noalloc_run(const float2* H, int32_t F, int32_t Nr, int32_t Nt,
                                const double* snr_db, int32_t n_snr, double* C, cudaStream_t s) {
    if (F > kNoAllocMaxF || n_snr > kNoAllocMaxSnr) {
        set_error("sbr_capacity_noalloc: F = %d and n_snr = %d exceed the fixed scratch (F <= %d, "
                  "n_snr <= %d); use sbr_capacity", F, n_snr, kNoAllocMaxF, kNoAllocMaxSnr);
        return SBR_ERR_INVALID_ARG;
    }
    CapacityScratch* scr = nullptr;
    SBR_TRY(capacity_scratch(&scr));
    // every scratch field read below is first written by this call, so nothing
    // has to be cleared; the SNR list travels by value in the launch itself
    SnrList snr{};
    for (int i = 0; i < n_snr; ++i) snr.lin[i] = std::pow(10.0, snr_db[i] / 10.0);
    ::sbr::note_launch(), k_snr_store<<<1, kMaxSnr, 0, s>>>(snr, n_snr, scr->snr_lin);
    ::sbr::note_launch(), k_frob<<<F, kCapThreads, 0, s>>>(H, (int64_t)Nr * Nt, scr->qf);
    ::sbr::note_launch(), k_qbar<<<1, 1, 0, s>>>(scr->qf, F, &scr->qbar);
    size_t smem = capacity_smem(Nr, Nt);
    SBR_TRY_CUDA(cudaFuncSetAttribute(k_capacity, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ::sbr::note_launch(), k_capacity<<<F, kCapThreads, smem, s>>>(H, Nr, Nt, scr->snr_lin, n_snr, &scr->qbar,
                                                                   scr->ld);
    ::sbr::note_launch(), k_cap_reduce<<<1, 32, 0, s>>>(scr->ld, F, n_snr, C);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

}  // namespace sbr
