// H(f) synthesis on the 5th-generation tensor cores (tcgen05), Eq. 13-14.
//
// For one frequency and the reflected paths n of one receiver,
//   H[q,p] = sum_n A[q,n] V[p,n],  A[q,n] = w_n exp(-j 2 pi f dr_qn / c),
//   V[p,n] = exp(-j 2 pi f dt_pn / c),
// is the complex contraction U diag(w) V^T. It runs as one real GEMM
//   C (2Nr x Nt) = A' (2Nr x 2P) B' (2P x Nt)
// with rows 2q / 2q+1 of C the real / imaginary part of H[q, :] and the
// contraction index k = 2n + {0: real, 1: imaginary}:
//   A'[2q,   2n] =  Re A,  A'[2q,   2n+1] = -Im A
//   A'[2q+1, 2n] =  Im A,  A'[2q+1, 2n+1] =  Re A
//   B'[2n, p]    =  Re V,  B'[2n+1, p]    =  Im V.
// Each operand is split x = hi + lo into two 16-bit values and the product is
// taken as hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory. Two
// forms: BF16 (the lo*lo term, ~2^-16 relative, dropped) and FP16 (~2^-22
// relative, with 5 exponent bits: A' is scaled per frequency by a power of two
// that brings max_n |w_n| into [1/2, 1), and the accumulator is scaled back,
// both exactly). The phasors are generated on chip
// (FP32 phase from the FP64-prepared delays) straight into 128-byte-swizzled
// K-major shared-memory tiles; one thread issues tcgen05.mma (M=128, N=256,
// K=16) and commits to an mbarrier; the epilogue reads TMEM with tcgen05.ld,
// pairs the real/imaginary rows across neighbouring lanes, adds the exact
// per-element LoS term and stores complex64.
//
// Every wait on the mbarrier is bounded; on expiry the CTA records
// ST_TIMEOUT, releases its tensor memory and returns.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "batch.cuh"
#include "tcgen05.cuh"
#include "sbr_internal.cuh"
#include "synth_common.cuh"

namespace sbr {
namespace {

using namespace tc;

constexpr int kTcThreads = 256;
constexpr int kChunkP = 32;      // paths per K-chunk (K = 64 16-bit values = one 128-byte row)
constexpr int kABytes = kTileM * 128;  // 16 KB: 2 x 64 receive elements

// tile of N transmit elements (N = 64, 128 or 256): shared-memory and TMEM sizes
template <int kTileN>
struct TcShape {
    static_assert(kTileN == 64 || kTileN == 128 || kTileN == 256, "tile N");
    static constexpr int kBBytes = kTileN * 128;
    static constexpr int kSmemTiles = 2 * kABytes + 2 * kBBytes;  // hi/lo of A and B
    static constexpr int kSmemBytes = kSmemTiles + 1024 + 64;      // + alignment slack + barriers
    static constexpr int kTmemCols = kTileN;                       // FP32 accumulator columns
};

// exp(-j 2 pi c) for a phase of c cycles: reduce to [-1/2, 1/2] exactly, then
// the hardware sine/cosine, whose absolute error on [-pi, pi] (below 1e-6) is
// well under the 2^-16 resolution of the BF16 hi/lo operands
__device__ __forceinline__ void phasor(float cycles, float& s, float& c) {
    float r = cycles - rintf(cycles);
    __sincosf(-6.283185307179586f * r, &s, &c);
}

// x = hi + lo, both BF16 or both FP16; returns the two as raw 16-bit patterns
template <bool kF16>
__device__ __forceinline__ void split16(float x, uint16_t& hi, uint16_t& lo) {
    if (kF16) {
        __half h = __float2half_rn(x);
        __half l = __float2half_rn(x - __half2float(h));
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(l);
    } else {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(l);
    }
}

struct TcArgs {
    // single receiver of one path list
    int32_t F, Nr, Nt;
    int32_t Pr;                // paths of the receiver (stride of w rows)
    const int32_t* nb0;        // reflections of the first path: 0 = LoS at local index 0
    const double* freqs;
    const float* dt;           // [Pr][Nt]
    const float* dr;           // [Pr][Nr]
    const float2* w;           // [F][Pr]
    const float* dlos;         // [Nr][Nt]
    float2* H;
    unsigned int* status;
    int inject_timeout;        // test-only: wait on a barrier nothing arrives at
    // batched form: items of all jobs of a wave
    const BatchJobDev* jobs;
    const int64_t* item_off;   // [n_jobs + 1] first item of each job
    int32_t n_jobs;
    int64_t items;
    const int32_t* np;         // [n_jobs] paths of each job
    const int32_t* nb;         // reflections per path slot (batch path store)
    int32_t path_cap;          // stride of a job's w rows
    const float* dt_all;
    const float* dr_all;
    const float* dl_all;
    const float2* w_all;
};

// one output tile: frequency f, receive elements [q0, q0 + 64), transmit
// elements [p0, p0 + N); reflected paths are the local indices
// [n0, n0 + nrefl); the LoS path, when present, is local index 0 and is added
// exactly in the epilogue
struct TcItem {
    int f, q0, p0, Nr, Nt, los, n0, nrefl;
    float foc;
    const float* dt;
    const float* dr;
    const float2* wf;          // weights of frequency f
    const float* dlos;
    float2* Hf;                // H of frequency f
};

template <bool kBatch, int kTileN>
__device__ __forceinline__ TcItem tc_item(const TcArgs& a, int64_t it) {
    TcItem x;
    int F, Pr;
    const int32_t* nb0;
    const double* freqs;
    const float2* w;
    float2* H;
    int64_t wstride;
    if (kBatch) {
        int lo = 0, hi = a.n_jobs - 1;   // the last job whose first item is <= it
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.item_off + mid) <= it) lo = mid; else hi = mid - 1;
        }
        const BatchJobDev* J = a.jobs + lo;
        it -= __ldg(a.item_off + lo);
        F = J->F; x.Nr = J->Nr; x.Nt = J->Nt;
        Pr = __ldg(a.np + lo);
        nb0 = a.nb + J->path_base;
        freqs = J->freqs;
        x.dt = a.dt_all + J->dt_base;
        x.dr = a.dr_all + J->dr_base;
        x.dlos = a.dl_all + J->dl_base;
        w = a.w_all + J->w_base;
        wstride = a.path_cap;
        H = J->H;
    } else {
        F = a.F; x.Nr = a.Nr; x.Nt = a.Nt;
        Pr = a.Pr;
        nb0 = a.nb0;
        freqs = a.freqs;
        x.dt = a.dt; x.dr = a.dr; x.dlos = a.dlos;
        w = a.w;
        wstride = a.Pr;
        H = a.H;
    }
    (void)F;
    const int mtiles = (x.Nr + 63) / 64, ntiles = (x.Nt + kTileN - 1) / kTileN;
    x.f = (int)(it / (mtiles * ntiles));
    const int rem = (int)(it - (int64_t)x.f * mtiles * ntiles);
    x.q0 = (rem / ntiles) * 64;
    x.p0 = (rem % ntiles) * kTileN;
    x.los = (Pr > 0 && *nb0 == 0) ? 0 : -1;
    x.n0 = x.los == 0 ? 1 : 0;
    x.nrefl = Pr - x.n0;
    x.foc = (float)(freqs[x.f] / kC0);
    x.wf = w + (int64_t)x.f * wstride;
    x.Hf = H + (int64_t)x.f * x.Nr * x.Nt;
    return x;
}

template <bool kF16, bool kBatch, int kTileN>
__global__ void __launch_bounds__(kTcThreads, 2) k_synth_tc(const __grid_constant__ TcArgs a) {
    using Sh = TcShape<kTileN>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float s_red[kTcThreads / 32];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA_hi = smem;
    unsigned char* sA_lo = smem + kABytes;
    unsigned char* sB_hi = smem + 2 * kABytes;
    unsigned char* sB_lo = smem + 2 * kABytes + Sh::kBBytes;
    uint64_t* mbar = (uint64_t*)(smem + Sh::kSmemTiles);
    uint64_t* never = (uint64_t*)(smem + Sh::kSmemTiles + 8);   // injected-fault barrier
    uint32_t* tmem_slot = (uint32_t*)(smem + Sh::kSmemTiles + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(Sh::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(never)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t mbar_a = smem_u32(mbar);
    uint32_t phase = 0;
    bool failed = false;
    // injected fault: the first phase of `never` never completes; the bounded
    // wait gives up and the CTA takes the same exit as a real timeout
    if (a.inject_timeout) failed = __syncthreads_or(!mbar_wait(smem_u32(never), 0u, 1u << 12)) != 0;

    const int64_t items = kBatch ? a.items
                                 : (int64_t)a.F * ((a.Nr + 63) / 64) * ((a.Nt + kTileN - 1) / kTileN);
    for (int64_t it = blockIdx.x; it < items && !failed; it += gridDim.x) {
        const TcItem x = tc_item<kBatch, kTileN>(a, it);
        const int nch = (x.nrefl + kChunkP - 1) / kChunkP;
        // FP16 form: power-of-two scale of this frequency's weights (exact)
        float sc = 1.f, isc = 1.f;
        if (kF16) {
            float m = 0.f;
            for (int n = x.n0 + tid; n < x.n0 + x.nrefl; n += kTcThreads) {
                float2 ww = __ldg(x.wf + n);
                m = fmaxf(m, fmaxf(fabsf(ww.x), fabsf(ww.y)));
            }
            for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) s_red[warp] = m;
            __syncthreads();
            m = s_red[0];
            for (int k = 1; k < kTcThreads / 32; ++k) m = fmaxf(m, s_red[k]);
            __syncthreads();  // s_red is rewritten for the next item
            if (m > 0.f) {
                int e;
                frexpf(m, &e);
                sc = ldexpf(1.f, -e);
                isc = ldexpf(1.f, e);
            }
        }
        for (int c = 0; c < nch && !failed; ++c) {
            const int nb = x.n0 + c * kChunkP;
            const int cnt = min(kChunkP, x.n0 + x.nrefl - nb);
            // A' tile: 64 receive elements x 32 paths, each a 2x2 real block;
            // consecutive threads take consecutive receive elements (coalesced)
#pragma unroll 4
            for (int e = tid; e < 64 * kChunkP; e += kTcThreads) {
                int ql = e & 63, nl = e >> 6;
                int q = x.q0 + ql, n = nb + nl;
                float ar = 0.f, ai = 0.f;
                if (nl < cnt && q < x.Nr) {
                    float2 ww = __ldg(x.wf + n);
                    float s, co;
                    phasor(x.foc * __ldg(x.dr + (int64_t)n * x.Nr + q), s, co);
                    ar = ww.x * co - ww.y * s;
                    ai = ww.x * s + ww.y * co;
                    if (kF16) { ar *= sc; ai *= sc; }
                }
                uint16_t h0, l0, h1, l1, h2, l2;
                split16<kF16>(ar, h0, l0);
                split16<kF16>(-ai, h1, l1);
                split16<kF16>(ai, h2, l2);
                uint32_t o0 = sw128(2 * ql, 2 * nl), o1 = sw128(2 * ql + 1, 2 * nl);
                *(uint32_t*)(sA_hi + o0) = (uint32_t)h0 | ((uint32_t)h1 << 16);
                *(uint32_t*)(sA_lo + o0) = (uint32_t)l0 | ((uint32_t)l1 << 16);
                *(uint32_t*)(sA_hi + o1) = (uint32_t)h2 | ((uint32_t)h0 << 16);
                *(uint32_t*)(sA_lo + o1) = (uint32_t)l2 | ((uint32_t)l0 << 16);
            }
            // B' tile (stored N x K): N transmit elements x 32 paths;
            // consecutive threads take consecutive transmit elements (coalesced)
#pragma unroll 8
            for (int e = tid; e < kTileN * kChunkP; e += kTcThreads) {
                int pl = e & (kTileN - 1), nl = e / kTileN;
                int p = x.p0 + pl, n = nb + nl;
                float vr = 0.f, vi = 0.f;
                if (nl < cnt && p < x.Nt) phasor(x.foc * __ldg(x.dt + (int64_t)n * x.Nt + p), vi, vr);
                uint16_t h0, l0, h1, l1;
                split16<kF16>(vr, h0, l0);
                split16<kF16>(vi, h1, l1);
                uint32_t o = sw128(pl, 2 * nl);
                *(uint32_t*)(sB_hi + o) = (uint32_t)h0 | ((uint32_t)h1 << 16);
                *(uint32_t*)(sB_lo + o) = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint64_t dAh = make_desc(smem_u32(sA_hi)), dAl = make_desc(smem_u32(sA_lo));
                uint64_t dBh = make_desc(smem_u32(sB_hi)), dBl = make_desc(smem_u32(sB_lo));
                for (int ks = 0; ks < 4; ++ks) {
                    uint64_t off = (uint64_t)(ks * 32) >> 4;  // 16 elements along K
                    mma_16<kF16, kTileN>(tmem, dAh + off, dBh + off, (c > 0 || ks > 0) ? 1u : 0u);
                    mma_16<kF16, kTileN>(tmem, dAh + off, dBl + off, 1u);
                    mma_16<kF16, kTileN>(tmem, dAl + off, dBh + off, 1u);
                }
                mma_commit(mbar_a);
            }
            const bool ok = mbar_wait(mbar_a, phase);
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            failed = __syncthreads_or(!ok) != 0;  // one decision for the whole CTA
        }
        if (failed) break;
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 and half (w / 4) of the N columns
        const int qw = warp & 3, chalf = warp >> 2;
        const int row = 32 * qw + lane;            // row of C: 2 (q - q0) + part
        const int q = x.q0 + (row >> 1);
        const int part = row & 1;
        float2 wl = make_float2(0.f, 0.f);
        if (x.los >= 0) wl = x.wf[x.los];
        for (int j = 0; j < kTileN / 64; ++j) {
            const int col0 = (kTileN / 2) * chalf + 32 * j;
            uint32_t v[32];
            if (nch > 0) {
                tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)col0, v);
            } else {
                for (int k = 0; k < 32; ++k) v[k] = 0u;
            }
            // even lane (real row) keeps columns [0,16), odd lane (imaginary row) [16,32)
            float re[16], im[16];
            for (int k = 0; k < 16; ++k) {
                float mine_lo = __uint_as_float(v[k]), mine_hi = __uint_as_float(v[16 + k]);
                float send = part == 0 ? mine_hi : mine_lo;
                float got = __shfl_xor_sync(0xffffffffu, send, 1);
                if (part == 0) { re[k] = mine_lo; im[k] = got; }
                else { re[k] = got; im[k] = mine_hi; }
                if (kF16) { re[k] *= isc; im[k] *= isc; }
            }
            const int pb = x.p0 + col0 + 16 * part;
            if (q < x.Nr) {
                float2* dst = x.Hf + (int64_t)q * x.Nt;
                if (x.los >= 0) {
                    float dl[16];
                    const float* src = x.dlos + (int64_t)q * x.Nt + pb;
                    if (pb + 16 <= x.Nt && ((((uintptr_t)src) & 15) == 0)) {
                        for (int k = 0; k < 4; ++k) {
                            float4 v4 = __ldg(reinterpret_cast<const float4*>(src) + k);
                            dl[4 * k] = v4.x; dl[4 * k + 1] = v4.y; dl[4 * k + 2] = v4.z; dl[4 * k + 3] = v4.w;
                        }
                    } else {
                        for (int k = 0; k < 16; ++k) dl[k] = pb + k < x.Nt ? __ldg(src + k) : 0.f;
                    }
                    for (int k = 0; k < 16; ++k) {
                        float s, co;
                        sincospif(-2.0f * x.foc * dl[k], &s, &co);
                        re[k] += wl.x * co - wl.y * s;
                        im[k] += wl.x * s + wl.y * co;
                    }
                }
                if (pb + 16 <= x.Nt && ((((uintptr_t)(dst + pb)) & 15) == 0)) {
                    float4* d4 = reinterpret_cast<float4*>(dst + pb);
                    for (int k = 0; k < 8; ++k)
                        d4[k] = make_float4(re[2 * k], im[2 * k], re[2 * k + 1], im[2 * k + 1]);
                } else {
                    for (int k = 0; k < 16 && pb + k < x.Nt; ++k) dst[pb + k] = make_float2(re[k], im[k]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (failed && tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::kTmemCols));
    }
}

// Operands of the tensor-core forms in one launch (the FP32 copies of the
// FP64 prologue of the CUDA-core forms): for the Pr paths of one receiver,
//   dt[n][p] = |T_p - P1| - |T_0 - P1|,  dr[n][q] = |R_q - Pm| - |R_0 - Pm|
//   (0 for the LoS path), dlos[q][p] = |T_p - R_q| - |T_0 - R_0| (FP64, then
//   rounded), and w[f][n] = g_n(f) exp(-j 2 pi frac(f L_n / c)) in FP64, then
//   rounded.
struct TcPrep {
    int32_t Pr, Nt, Nr, F;
    const int32_t* nb;       // [Pr] reflections of the receiver's paths
    const double* pts;       // [Pr][kKmax][3]
    const double* L;         // [Pr]
    const float2* g;         // [Pr][F]
    const double* freqs;
    const double* tx_elem;
    const double* rx_elem;
    const double* R0;
    d3 T0;
    float* dt;
    float* dr;
    float* dlos;
    float2* w;
};

__global__ void k_tc_prep(const __grid_constant__ TcPrep a) {
    const int64_t n_dt = (int64_t)a.Pr * a.Nt, n_dr = (int64_t)a.Pr * a.Nr, n_dl = (int64_t)a.Nr * a.Nt;
    const int64_t total = n_dt + n_dr + n_dl + (int64_t)a.F * a.Pr;
    const d3 R0 = ld3(a.R0);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n_dt) {
            const int64_t n = t / a.Nt;
            const int p = (int)(t - n * a.Nt);
            float v = 0.f;
            if (a.nb[n] > 0) {
                const d3 P1 = ld3(a.pts + n * kKmax * 3);
                v = (float)(norm(ld3(a.tx_elem + 3 * p) - P1) - norm(a.T0 - P1));
            }
            a.dt[t] = v;
        } else if (t < n_dt + n_dr) {
            const int64_t u = t - n_dt, n = u / a.Nr;
            const int q = (int)(u - n * a.Nr);
            const int m = a.nb[n];
            float v = 0.f;
            if (m > 0) {
                const d3 Pm = ld3(a.pts + (n * kKmax + m - 1) * 3);
                v = (float)(norm(ld3(a.rx_elem + 3 * q) - Pm) - norm(R0 - Pm));
            }
            a.dr[u] = v;
        } else if (t < n_dt + n_dr + n_dl) {
            const int64_t u = t - n_dt - n_dr, q = u / a.Nt;
            const int p = (int)(u - q * a.Nt);
            a.dlos[u] = (float)(norm(ld3(a.tx_elem + 3 * p) - ld3(a.rx_elem + 3 * q)) - norm(a.T0 - R0));
        } else {
            const int64_t u = t - n_dt - n_dr - n_dl, f = u / a.Pr, n = u - f * a.Pr;
            // the batched form computes its weights with the same FP64 arithmetic,
            // so both give bit-identical H for the same path list
            const double cyc = a.freqs[f] * a.L[n] / kC0;
            const double frc = cyc - floor(cyc);
            double s, c;
            sincospi(-2.0 * frc, &s, &c);
            const float2 gg = a.g[n * a.F + f];
            a.w[u] = make_float2((float)(gg.x * c - gg.y * s), (float)(gg.x * s + gg.y * c));
        }
    }
}

inline unsigned nb256(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

}  // namespace

sbr_status synth_tc_run(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                        const double* tx_elem, int32_t Nt, const double* rx_elem, int32_t Nr,
                        int32_t rx_index, float2* H, bool f16, cudaStream_t s) {
    const int32_t o0 = pl->h_rx_off[rx_index], Pr_ = pl->h_rx_off[rx_index + 1] - o0;
    const int32_t Pr = std::max(Pr_, 1);
    // one buffer for the four operands: w (8-byte elements) first
    const size_t n_w = (size_t)Pr * F, n_f = (size_t)Pr * Nt + (size_t)Pr * Nr + (size_t)Nr * Nt;
    float2* w;
    SBR_TRY(dalloc_n(&w, n_w + (n_f + 1) / 2, s));
    float* dt = reinterpret_cast<float*>(w + n_w);
    float* dr = dt + (size_t)Pr * Nt;
    float* dl = dr + (size_t)Pr * Nr;
    TcPrep pp{};
    pp.Pr = Pr_; pp.Nt = Nt; pp.Nr = Nr; pp.F = F;
    pp.nb = pl->nb + o0;
    pp.pts = pl->pts + (int64_t)o0 * kKmax * 3;
    pp.L = pl->L + o0;
    pp.g = g + (int64_t)o0 * F;
    pp.freqs = freqs; pp.tx_elem = tx_elem; pp.rx_elem = rx_elem;
    pp.R0 = pl->rx_xyz + 3 * rx_index;
    pp.T0 = mk3(pl->tx[0], pl->tx[1], pl->tx[2]);
    pp.dt = dt; pp.dr = dr; pp.dlos = dl; pp.w = w;
    const int64_t n_all = (int64_t)Pr_ * (Nt + Nr) + (int64_t)Nr * Nt + (int64_t)Pr_ * F;
    ::sbr::note_launch(), k_tc_prep<<<(unsigned)std::min<int64_t>(nb256(n_all), 8 * (int64_t)sm_count()), 256, 0, s>>>(pp);
    SBR_TRY_CUDA(cudaGetLastError());
    TcArgs a{};
    a.F = F; a.Nr = Nr; a.Nt = Nt;
    a.Pr = Pr_;
    a.nb0 = pl->nb + o0;
    a.freqs = freqs; a.dt = dt; a.dr = dr; a.w = w; a.dlos = dl; a.H = H;
    a.status = pl->d_status;  // a bounded wait that gave up is reported by sbr_path_query
    a.inject_timeout = fault_mode() == kFaultTimeout ? 1 : 0;
    auto kern = f16 ? k_synth_tc<true, false, 256> : k_synth_tc<false, false, 256>;
    constexpr int kSmemBytes = TcShape<256>::kSmemBytes;
    SBR_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    int64_t items = (int64_t)F * ((Nr + 63) / 64) * ((Nt + 255) / 256);
    // two CTAs per SM (97 KB shared memory and 256 TMEM columns each): one CTA's
    // MMA and epilogue overlap the other's phasor generation
    int grid = (int)std::min<int64_t>(items, 2 * (int64_t)sm_count());
    ::sbr::note_launch(), kern<<<grid, kTcThreads, kSmemBytes, s>>>(a);
    SBR_TRY_CUDA(cudaGetLastError());
    dfree(w, s);
    return SBR_OK;
}

namespace {
template <bool kF16, int kTileN>
sbr_status batch_tc_launch(const BatchSynthWave& w, cudaStream_t s) {
    TcArgs a{};
    a.jobs = w.jobs;
    a.item_off = w.item_off;
    a.n_jobs = w.n_jobs;
    a.items = w.items;
    a.np = w.np;
    a.nb = w.nb;
    a.path_cap = w.path_cap;
    a.dt_all = w.dt;
    a.dr_all = w.dr;
    a.dl_all = w.dl;
    a.w_all = w.w;
    a.status = w.status;
    a.inject_timeout = fault_mode() == kFaultTimeout ? 1 : 0;
    if (w.items <= 0) return SBR_OK;
    int grid = (int)std::min<int64_t>(w.items, 2 * (int64_t)sm_count());
    ::sbr::note_launch(), k_synth_tc<kF16, true, kTileN><<<grid, kTcThreads, TcShape<kTileN>::kSmemBytes, s>>>(a);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

template <bool kF16, int kTileN>
sbr_status batch_tc_attr() {
    SBR_TRY_CUDA(cudaFuncSetAttribute(k_synth_tc<kF16, true, kTileN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TcShape<kTileN>::kSmemBytes));
    return SBR_OK;
}
}  // namespace

sbr_status batch_synth_prepare(bool f16, int tile_n) {
    switch (tile_n) {
        case 64: return f16 ? batch_tc_attr<true, 64>() : batch_tc_attr<false, 64>();
        case 128: return f16 ? batch_tc_attr<true, 128>() : batch_tc_attr<false, 128>();
        case 256: return f16 ? batch_tc_attr<true, 256>() : batch_tc_attr<false, 256>();
        default: set_error("tile_n %d not in {64, 128, 256}", tile_n); return SBR_ERR_INVALID_ARG;
    }
}

sbr_status batch_synth_tc(const BatchSynthWave& w, bool f16, int tile_n, cudaStream_t s) {
    switch (tile_n) {
        case 64: return f16 ? batch_tc_launch<true, 64>(w, s) : batch_tc_launch<false, 64>(w, s);
        case 128: return f16 ? batch_tc_launch<true, 128>(w, s) : batch_tc_launch<false, 128>(w, s);
        case 256: return f16 ? batch_tc_launch<true, 256>(w, s) : batch_tc_launch<false, 256>(w, s);
        default: set_error("tile_n %d not in {64, 128, 256}", tile_n); return SBR_ERR_INVALID_ARG;
    }
}

}  // namespace sbr
