// H(f) synthesis on the 5th-generation tensor cores (tcgen05), Eq. 13-14.
//
// For one frequency and the reflected paths n of one receiver,
//   H[q,p] = sum_n A[q,n] V[p,n],  A[q,n] = w_n exp(-j 2 pi f dr_qn / c),
//   V[p,n] = exp(-j 2 pi f dt_pn / c),
// is the complex contraction U diag(w) V^T. It runs as one real GEMM
//   C (2Nr x Nt) = A' (2Nr x 2P) B' (2P x Nt)
// with rows r(q) / i(q) of C the real / imaginary part of H[q, :] and the
// contraction index k = 2n + {0: real, 1: imaginary}:
//   A'[r(q), 2n] =  Re A,  A'[r(q), 2n+1] = -Im A
//   A'[i(q), 2n] =  Im A,  A'[i(q), 2n+1] =  Re A
//   B'[2n, p]    =  Re V,  B'[2n+1, p]    =  Im V;
// in a tile of 64 receive elements, r(q) = 16 (q / 8) + q % 8 and
// i(q) = r(q) + 8 (acc_row).
// Each operand is split x = hi + lo into two 16-bit values and the product is
// taken as hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory. Two
// forms: BF16 (the lo*lo term, ~2^-16 relative, dropped) and FP16 (~2^-22
// relative, with 5 exponent bits: A' is scaled per frequency by a power of two
// that brings max_n |w_n| into [1/2, 1), and the accumulator is scaled back,
// both exactly). The phasors are generated on chip
// (FP32 phase from the FP64-prepared delays) straight into 128-byte-swizzled
// K-major shared-memory tiles; one thread issues tcgen05.mma (M=128, N=256,
// K=16) and commits to an mbarrier; the epilogue reads TMEM with tcgen05.ld
// in the 16-lane shape that gives each thread the real and the imaginary row
// of one receive element, adds the exact per-element LoS term and stores
// complex64.
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
#include "synth_ops.cuh"

namespace sbr {
namespace {

using namespace tc;

constexpr int kTcThreads = 512;  // 16 warps, one CTA per SM
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kChunkP = 32;      // paths per K-chunk (K = 64 16-bit values = one 128-byte row)
constexpr int kABytes = kTileM * 128;  // 16 KB: 2 x 64 receive elements

// tile of N transmit elements (N = 64, 128 or 256): shared-memory and TMEM sizes.
// Two operand stages (hi/lo of A' and B' each) and two FP32 accumulators, so
// that the phasors of one K-chunk are generated while the tensor core works on
// the previous one and a tile's epilogue runs while the next tile's MMAs do.
template <int kTileN>
struct TcShape {
    static_assert(kTileN == 64 || kTileN == 128 || kTileN == 256, "tile N");
    static constexpr int kBBytes = kTileN * 128;
    static constexpr int kStage = 2 * kABytes + 2 * kBBytes;        // hi/lo of A and B
    static constexpr int kSmemBytes = 2 * kStage + 1024 + 128;      // + alignment + barriers
    static constexpr int kTmemCols = 2 * kTileN;                    // two accumulators
};

// exp(-j 2 pi c) for a phase of c cycles: reduce to [-1/2, 1/2] exactly, then
// the hardware sine/cosine, whose absolute error on [-pi, pi] (below 1e-6) is
// well under the 2^-16 resolution of the BF16 hi/lo operands
__device__ __forceinline__ void phasor(float cycles, float& s, float& c) {
    float r = cycles - rintf(cycles);
    __sincosf(-6.283185307179586f * r, &s, &c);
}

// Operands of the tensor-core forms (layouts in synth_ops.cuh): reflected
// paths only, transposed and padded to Pp (a multiple of 8) paths per row, so
// that four paths of one element are one 16-byte load; the LoS weight and the
// FP16 scale per frequency come separately.
struct TcArgs {
    // single receiver of one path list
    int32_t F, Nr, Nt;
    int32_t Pr;                // paths of the receiver (LoS included)
    int32_t Pp;                // padded row length of dtT, drT and w
    const int32_t* nb0;        // reflections of the first path: 0 = it is the LoS path
    const double* freqs;
    const float* dtT;          // [Pp/4][Nt][4]
    const float* drT;          // [Pp/4][Nr][4]
    const float2* w;           // [F][Pp]
    const float2* wl;          // [F]
    const float* sc;           // [F]
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
    int32_t path_cap;          // padded row length of a job's operands
    const float* dt_all;
    const float* dr_all;
    const float* dl_all;
    const float2* w_all;
    const float2* wl_all;
    const float* sc_all;
};

// one output tile: frequency f, receive elements [q0, q0 + 64), transmit
// elements [p0, p0 + N); the reflected paths [0, nrefl) go through the tensor
// cores, the LoS path (if any) is added exactly in the epilogue
struct TcItem {
    int f, q0, p0, Nr, Nt, nrefl, Pp;
    bool los;
    float foc, sc;
    float2 wl;
    const float* dtT;
    const float* drT;
    const float2* wf;          // reflected-path weights of frequency f
    const float* dlos;
    float2* Hf;                // H of frequency f
};

template <bool kBatch, int kTileN>
__device__ __forceinline__ TcItem tc_item(const TcArgs& a, int64_t it) {
    TcItem x;
    int Pr;
    const int32_t* nb0;
    const double* freqs;
    const float2* w;
    const float2* wl;
    const float* sc;
    float2* H;
    if (kBatch) {
        int lo = 0, hi = a.n_jobs - 1;   // the last job whose first item is <= it
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.item_off + mid) <= it) lo = mid; else hi = mid - 1;
        }
        const BatchJobDev* J = a.jobs + lo;
        it -= __ldg(a.item_off + lo);
        x.Nr = J->Nr; x.Nt = J->Nt;
        Pr = __ldg(a.np + lo);
        nb0 = a.nb + J->path_base;
        freqs = J->freqs;
        x.dtT = a.dt_all + J->dt_base;
        x.drT = a.dr_all + J->dr_base;
        x.dlos = a.dl_all + J->dl_base;
        w = a.w_all + J->w_base;
        wl = a.wl_all + J->wl_base;
        sc = a.sc_all + J->wl_base;
        x.Pp = a.path_cap;
        H = J->H;
    } else {
        x.Nr = a.Nr; x.Nt = a.Nt;
        Pr = a.Pr;
        nb0 = a.nb0;
        freqs = a.freqs;
        x.dtT = a.dtT; x.drT = a.drT; x.dlos = a.dlos;
        w = a.w;
        wl = a.wl;
        sc = a.sc;
        x.Pp = a.Pp;
        H = a.H;
    }
    // 32-bit decode (a job has F * tiles < 2^31 items); every thread of the
    // CTA repeats it, so it stays cheap
    const uint32_t mtiles = (uint32_t)(x.Nr + 63) / 64u, ntiles = (uint32_t)(x.Nt + kTileN - 1) / (uint32_t)kTileN;
    const uint32_t per_f = mtiles * ntiles, itu = (uint32_t)it;
    const uint32_t fq = per_f == 1u ? itu : itu / per_f;
    const uint32_t rem = itu - fq * per_f;
    const uint32_t qt = ntiles == 1u ? rem : rem / ntiles;
    x.f = (int)fq;
    x.q0 = (int)qt * 64;
    x.p0 = (int)(rem - qt * ntiles) * kTileN;
    x.los = Pr > 0 && *nb0 == 0;
    x.nrefl = Pr - (x.los ? 1 : 0);
    x.foc = (float)(freqs[x.f] * kInvC0);
    x.wf = w + (int64_t)x.f * x.Pp;
    x.wl = wl[x.f];
    x.sc = sc[x.f];
    x.Hf = H + (int64_t)x.f * x.Nr * x.Nt;
    return x;
}

// x = hi + lo for a pair of values, both BF16 or both FP16: the hi and lo
// halves of two K positions packed as two 32-bit words (lower K index in the
// low 16 bits)
template <bool kF16>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    if (kF16) {
        __half2 h = __floats2half2_rn(x0, x1);
        float2 hf = __half22float2(h);
        __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<uint32_t*>(&h);
        lo = *reinterpret_cast<uint32_t*>(&l);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        float2 hf = __bfloat1622float2(h);
        __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<uint32_t*>(&h);
        lo = *reinterpret_cast<uint32_t*>(&l);
    }
}

// byte offset of the 16-byte chunk c (8 K values) of row r in a 128-byte
// swizzled K-major tile (the layout the matrix descriptors describe)
__device__ __forceinline__ uint32_t chunk_off(int r, int c) {
    return (uint32_t)r * 128u + ((uint32_t)(c ^ (r & 7)) << 4);
}

// shared-memory store without a compiler memory barrier: global loads of later
// work may be hoisted above it (the stores stay ordered among the volatile
// statements, and the tensor core reads them only after a proxy fence and a
// barrier)
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d));
}

// what the epilogue of a tile needs once its MMAs have been issued
struct TcEpi {
    int q0, p0, Nr, Nt, acc;
    bool los;
    bool full;                 // whole tile inside H, even Nt, aligned rows: no per-output checks
    bool mma;                  // the tile has reflected paths (an accumulator to read)
    uint32_t acc_parity;       // phase of acc_full[acc] that completes this tile
    float foc, isc;
    float2 wl;                 // LoS weight (unscaled)
    const float* dlos;
    float2* Hf;
};

// Row of the M = 128 accumulator that holds the real (part 0) or imaginary
// (part 1) part of receive element ql of the tile: receive elements come in
// groups of 8, their real rows followed by their imaginary rows, so that one
// 16-lane tensor-memory load hands each thread both parts of one output
__device__ __forceinline__ int acc_row(int ql, int part) { return 16 * (ql >> 3) + 8 * part + (ql & 7); }

// Epilogue of one tile: warp w reads TMEM lanes [32 (w % 4), + 32) (receive
// elements [16 (w % 4), + 16) of the tile) over its N / 4 columns, 16 lanes
// (8 receive elements) x 32 columns at a time; thread t receives, for 8
// consecutive columns, (Re, Im) of receive element t / 4 at transmit elements
// 2 (t % 4) and + 1. It scales back (FP16 form), adds the exact per-element
// LoS term and writes them as one 16-byte store (four lanes write 64
// contiguous bytes of a row of H).
template <bool kF16, int kTileN>
__device__ __forceinline__ void tc_epilogue(const TcEpi& e, uint32_t tmem, int warp, int lane) {
    const int lg = warp & 3, cg = warp >> 2;   // TMEM lane quarter, column group
    constexpr int kCols = kTileN / 4;          // columns of one warp
    constexpr int kRep = kCols >= 32 ? 4 : kCols / 8;   // 8-column repeats per load
    constexpr int kBlkCols = 8 * kRep;
    constexpr int kJ = kCols / kBlkCols;       // column blocks per 16-lane half
    constexpr int kBlocks = 2 * kJ;
    const int qa = lane >> 2, pc = 2 * (lane & 3);
    const uint32_t tacc = tmem + (uint32_t)(e.acc * kTileN);
    if (e.full) {
        // every output of the tile exists: no per-output checks. 32-bit element
        // offsets within frequency f's H and LoS delays (Nr * Nt < 2^31 for a
        // full tile); the LoS delays of block b + 1 are requested while block b
        // is processed
        auto offset = [&](int b, int k) {
            const int h = b / kJ, jj = b % kJ;
            const uint32_t q = (uint32_t)(e.q0 + 16 * lg + 8 * h + qa);
            return q * (uint32_t)e.Nt + (uint32_t)(e.p0 + cg * kCols + kBlkCols * jj + 8 * k + pc);
        };
        float2 dl_next[kRep];
        if (e.los) {
#pragma unroll
            for (int k = 0; k < kRep; ++k) dl_next[k] = __ldg(reinterpret_cast<const float2*>(e.dlos + offset(0, k)));
        }
#pragma unroll
        for (int b = 0; b < kBlocks; ++b) {
            const int h = b / kJ, jj = b % kJ;
            float2 dl[kRep];
            if (e.los) {
#pragma unroll
                for (int k = 0; k < kRep; ++k) dl[k] = dl_next[k];
                if (b + 1 < kBlocks) {
#pragma unroll
                    for (int k = 0; k < kRep; ++k)
                        dl_next[k] = __ldg(reinterpret_cast<const float2*>(e.dlos + offset(b + 1, k)));
                }
            }
            uint32_t v[4 * kRep];
            if (e.mma) {
                tmem_ld_16x256b<kRep>(tacc + ((uint32_t)(32 * lg + 16 * h) << 16) + (uint32_t)(cg * kCols + kBlkCols * jj), v);
            } else {
#pragma unroll
                for (int k = 0; k < 4 * kRep; ++k) v[k] = 0u;
            }
#pragma unroll
            for (int k = 0; k < kRep; ++k) {
                const float re0 = __uint_as_float(v[4 * k]), re1 = __uint_as_float(v[4 * k + 1]);
                const float im0 = __uint_as_float(v[4 * k + 2]), im1 = __uint_as_float(v[4 * k + 3]);
                float4 o = kF16 ? make_float4(re0 * e.isc, im0 * e.isc, re1 * e.isc, im1 * e.isc)
                                : make_float4(re0, im0, re1, im1);
                if (e.los) {
                    float sn, cs;
                    phasor(e.foc * dl[k].x, sn, cs);
                    o.x = fmaf(e.wl.x, cs, fmaf(-e.wl.y, sn, o.x));
                    o.y = fmaf(e.wl.x, sn, fmaf(e.wl.y, cs, o.y));
                    phasor(e.foc * dl[k].y, sn, cs);
                    o.z = fmaf(e.wl.x, cs, fmaf(-e.wl.y, sn, o.z));
                    o.w = fmaf(e.wl.x, sn, fmaf(e.wl.y, cs, o.w));
                }
                *reinterpret_cast<float4*>(e.Hf + offset(b, k)) = o;
            }
        }
        return;
    }
#pragma unroll 1
    for (int b = 0; b < kBlocks; ++b) {
        const int h = b / kJ, jj = b % kJ;
        const int q = e.q0 + 16 * lg + 8 * h + qa;
        const int pb = e.p0 + cg * kCols + kBlkCols * jj + pc;
        // LoS delays of this lane's outputs, requested before the tensor-memory
        // load so that their latency overlaps it
        float2 dl[kRep];
#pragma unroll
        for (int k = 0; k < kRep; ++k) {
            const int p = pb + 8 * k;
            dl[k] = make_float2(0.f, 0.f);
            if (e.los && q < e.Nr && p < e.Nt) {
                const float* src = e.dlos + (int64_t)q * e.Nt + p;
                if (p + 1 < e.Nt && ((((uintptr_t)src) & 7) == 0)) dl[k] = __ldg(reinterpret_cast<const float2*>(src));
                else dl[k] = make_float2(__ldg(src), p + 1 < e.Nt ? __ldg(src + 1) : 0.f);
            }
        }
        uint32_t v[4 * kRep];
        if (e.mma) {
            tmem_ld_16x256b<kRep>(tacc + ((uint32_t)(32 * lg + 16 * h) << 16) + (uint32_t)(cg * kCols + kBlkCols * jj), v);
        } else {
#pragma unroll
            for (int k = 0; k < 4 * kRep; ++k) v[k] = 0u;
        }
#pragma unroll
        for (int k = 0; k < kRep; ++k) {
            const int p = pb + 8 * k;
            const float re0 = __uint_as_float(v[4 * k]), re1 = __uint_as_float(v[4 * k + 1]);
            const float im0 = __uint_as_float(v[4 * k + 2]), im1 = __uint_as_float(v[4 * k + 3]);
            float4 o = make_float4(re0 * e.isc, im0 * e.isc, re1 * e.isc, im1 * e.isc);
            if (e.los) {
                float sn, cs;
                phasor(e.foc * dl[k].x, sn, cs);
                o.x = fmaf(e.wl.x, cs, fmaf(-e.wl.y, sn, o.x));
                o.y = fmaf(e.wl.x, sn, fmaf(e.wl.y, cs, o.y));
                phasor(e.foc * dl[k].y, sn, cs);
                o.z = fmaf(e.wl.x, cs, fmaf(-e.wl.y, sn, o.z));
                o.w = fmaf(e.wl.x, sn, fmaf(e.wl.y, cs, o.w));
            }
            if (q < e.Nr && p < e.Nt) {
                float2* dst = e.Hf + (int64_t)q * e.Nt + p;
                if (p + 1 < e.Nt && ((((uintptr_t)dst) & 15) == 0)) {
                    *reinterpret_cast<float4*>(dst) = o;
                } else {
                    dst[0] = make_float2(o.x, o.y);
                    if (p + 1 < e.Nt) dst[1] = make_float2(o.z, o.w);
                }
            }
        }
    }
}

template <bool kF16, bool kBatch, int kTileN>
__global__ void __launch_bounds__(kTcThreads, 1) k_synth_tc(const __grid_constant__ TcArgs a) {
    using Sh = TcShape<kTileN>;
    static_assert(kTcThreads % kTileN == 0 && 64 * (kChunkP / 4) <= kTcThreads, "generation units");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + 2 * Sh::kStage);
    // bars: mma_done[0..1] (per operand stage), acc_full[0..1] (per accumulator),
    // never (injected fault), drain (final wait before the tensor memory is freed)
    const uint32_t bar0 = smem_u32(bars);
    auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    uint32_t* tmem_slot = (uint32_t*)(bars + 6);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(Sh::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 6; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(i)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // launched as a programmatic dependent of the operand prologue, the
    // prologue above overlaps its tail; its results are read only after this
    // (a no-op for an ordinary launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    bool failed = false;
    // injected fault: the first phase of `never` never completes; the bounded
    // wait gives up and the CTA takes the same exit as a real timeout
    if (a.inject_timeout) failed = __syncthreads_or(!mbar_wait(bar(4), 0u, 1u << 12)) != 0;

    const int64_t items = kBatch ? a.items
                                 : (int64_t)a.F * ((a.Nr + 63) / 64) * ((a.Nt + kTileN - 1) / kTileN);
    uint32_t stage_uses0 = 0u, stage_uses1 = 0u;   // chunks issued per operand stage
    uint32_t acc_uses0 = 0u, acc_uses1 = 0u;       // tiles with MMAs per accumulator
    uint32_t chunk_all = 0;
    TcEpi prev{};
    bool have_prev = false;
    bool epi_ok = true;   // this thread's last epilogue wait succeeded (folded into the next barrier)
    int local = 0;
    for (int64_t it = blockIdx.x; it < items && !failed; it += gridDim.x, ++local) {
        const TcItem x = tc_item<kBatch, kTileN>(a, it);
        const int acc = local & 1;
        const int nch = (x.nrefl + kChunkP - 1) / kChunkP;
        // FP16 form: the power-of-two scale of this frequency's weights (exact)
        const float sc = kF16 ? x.sc : 1.f;
        for (int c = 0; c < nch; ++c) {
            const int st = chunk_all & 1;
            unsigned char* sA_hi = smem + st * Sh::kStage;
            unsigned char* sA_lo = sA_hi + kABytes;
            unsigned char* sB_hi = sA_hi + 2 * kABytes;
            unsigned char* sB_lo = sB_hi + Sh::kBBytes;
            bool ok = true;
            // the stage is free once the MMAs of its previous chunk have completed
            const uint32_t su = st ? stage_uses1 : stage_uses0;
            if (su > 0) ok = mbar_wait(bar(st), (su - 1u) & 1u);
            const int nb = c * kChunkP;
            const int cnt = min(kChunkP, x.nrefl - nb);
            const int nks = (cnt + 7) >> 3;        // MMA K-steps (8 paths each)
            const int n16 = 2 * nks;               // 16-byte chunks per row (4 paths each)
            if (ok) {
                // B' (stored N x K): transmit element p, paths nb + 4 c16 .. + 3
                // (padded paths have zero weight, so their phasors are harmless);
                // kTcThreads is a multiple of N, so a thread keeps its element and
                // steps through the chunks
                {
                    const int pl = tid % kTileN;
                    const int p = x.p0 + pl;
                    // [Pp / 4][Nt] groups of 4 paths: consecutive lanes read
                    // consecutive 16-byte groups
                    const float4* src = reinterpret_cast<const float4*>(x.dtT) + (int64_t)(nb >> 2) * x.Nt + (p < x.Nt ? p : 0);
                    const uint32_t b_hi = smem_u32(sB_hi) + (uint32_t)pl * 128u;
                    const uint32_t b_lo = smem_u32(sB_lo) + (uint32_t)pl * 128u;
#pragma unroll 2
                    for (int c16 = tid / kTileN; c16 < n16; c16 += kTcThreads / kTileN) {
                        float4 d4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (p < x.Nt) d4 = __ldg(src + (int64_t)c16 * x.Nt);
                        float vr[4], vi[4];
                        phasor(x.foc * d4.x, vi[0], vr[0]);
                        phasor(x.foc * d4.y, vi[1], vr[1]);
                        phasor(x.foc * d4.z, vi[2], vr[2]);
                        phasor(x.foc * d4.w, vi[3], vr[3]);
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) split2<kF16>(vr[k], vi[k], h[k], l[k]);
                        const uint32_t o = (uint32_t)(c16 ^ (pl & 7)) << 4;   // chunk_off(pl, c16) - pl * 128
                        sts128(b_hi + o, h[0], h[1], h[2], h[3]);
                        sts128(b_lo + o, l[0], l[1], l[2], l[3]);
                    }
                }
                // A': receive element q, paths nb + 4 c16 .. + 3, as the two rows
                // r(q) (Re A, -Im A) and i(q) (Im A, Re A); consecutive lanes take
                // consecutive receive elements (rows r(q) & 7 = q & 7), so that a
                // quarter warp's 16-byte stores land in 8 distinct bank groups of
                // the swizzled rows and a warp shares its weights (at most 64 x 8
                // units: one per thread)
                const int v = tid;
                if (v < 64 * n16) {
                    const int ql = v & 63, c16 = v >> 6;
                    const int q = x.q0 + ql;
                    const int n = nb + 4 * c16;
                    float4 d4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 w01 = d4, w23 = d4;
                    if (q < x.Nr) {
                        d4 = __ldg(reinterpret_cast<const float4*>(x.drT) + (int64_t)(n >> 2) * x.Nr + q);
                        w01 = __ldg(reinterpret_cast<const float4*>(x.wf + n));
                        w23 = __ldg(reinterpret_cast<const float4*>(x.wf + n + 2));
                    }
                    const float dd[4] = {d4.x, d4.y, d4.z, d4.w};
                    const float wr[4] = {w01.x, w01.z, w23.x, w23.z};
                    const float wi[4] = {w01.y, w01.w, w23.y, w23.w};
                    uint32_t h0[4], l0[4], h1[4], l1[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float sn, cs;
                        phasor(x.foc * dd[k], sn, cs);
                        const float ar = (wr[k] * cs - wi[k] * sn) * sc;
                        const float ai = (wr[k] * sn + wi[k] * cs) * sc;
                        split2<kF16>(ar, -ai, h0[k], l0[k]);
                        // row i(q) holds (Im A, Re A): the same halves swapped, with
                        // the sign of -Im A flipped (rounding to nearest is symmetric,
                        // so these are the bits of a split of (ai, ar))
                        h1[k] = __byte_perm(h0[k], 0u, 0x1032) ^ 0x8000u;
                        l1[k] = __byte_perm(l0[k], 0u, 0x1032) ^ 0x8000u;
                    }
                    const uint32_t o0 = chunk_off(acc_row(ql, 0), c16), o1 = chunk_off(acc_row(ql, 1), c16);
                    sts128(smem_u32(sA_hi) + o0, h0[0], h0[1], h0[2], h0[3]);
                    sts128(smem_u32(sA_lo) + o0, l0[0], l0[1], l0[2], l0[3]);
                    sts128(smem_u32(sA_hi) + o1, h1[0], h1[1], h1[2], h1[3]);
                    sts128(smem_u32(sA_lo) + o1, l1[0], l1[1], l1[2], l1[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            // one decision for the whole CTA (this chunk's wait and the last epilogue's)
            failed = __syncthreads_or(!(ok && epi_ok)) != 0;
            if (failed) break;
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dAh = make_desc(smem_u32(sA_hi)), dAl = make_desc(smem_u32(sA_lo));
                const uint64_t dBh = make_desc(smem_u32(sB_hi)), dBl = make_desc(smem_u32(sB_lo));
                const uint32_t d = tmem + (uint32_t)(acc * kTileN);
                for (int ks = 0; ks < nks; ++ks) {
                    const uint64_t off = (uint64_t)(ks * 32) >> 4;  // 16 K values
                    mma_16<kF16, kTileN>(d, dAh + off, dBh + off, (c > 0 || ks > 0) ? 1u : 0u);
                    mma_16<kF16, kTileN>(d, dAh + off, dBl + off, 1u);
                    mma_16<kF16, kTileN>(d, dAl + off, dBh + off, 1u);
                }
                mma_commit(bar(st));
                if (c == nch - 1) mma_commit(bar(2 + acc));
            }
            if (st) stage_uses1 += 1u; else stage_uses0 += 1u;
            chunk_all += 1u;
        }
        if (failed) break;
        TcEpi cur;
        cur.q0 = x.q0; cur.p0 = x.p0; cur.Nr = x.Nr; cur.Nt = x.Nt; cur.los = x.los; cur.acc = acc;
        cur.mma = nch > 0;
        cur.acc_parity = (acc ? acc_uses1 : acc_uses0) & 1u;
        if (nch > 0) {
            if (acc) acc_uses1 += 1u; else acc_uses0 += 1u;
        }
        cur.foc = x.foc;
        cur.isc = kF16 ? 1.f / sc : 1.f;   // exact: sc is a power of two
        cur.wl = x.wl;
        cur.dlos = x.dlos; cur.Hf = x.Hf;
        cur.full = x.q0 + 64 <= x.Nr && x.p0 + kTileN <= x.Nt && (x.Nt & 1) == 0 &&
                   (int64_t)x.Nr * x.Nt < ((int64_t)1 << 31) &&   // 32-bit offsets in the fast epilogue
                   ((((uintptr_t)x.Hf) & 15) == 0) && (!x.los || ((((uintptr_t)x.dlos) & 7) == 0));
        // the previous tile's epilogue runs while this tile's MMAs do; no
        // barrier follows it: the next tile's first chunk barrier carries its
        // status, and its accumulator is written again only after that barrier
        if (have_prev) {
            bool ok = true;
            if (prev.mma) {
                ok = __all_sync(0xffffffffu, mbar_wait(bar(2 + prev.acc), prev.acc_parity));
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            if (ok) tc_epilogue<kF16, kTileN>(prev, tmem, warp, lane);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            epi_ok = epi_ok && ok;
        }
        prev = cur;
        have_prev = true;
    }
    if (!failed && have_prev) {
        bool ok = true;
        if (prev.mma) {
            ok = __all_sync(0xffffffffu, mbar_wait(bar(2 + prev.acc), prev.acc_parity));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        if (ok) tc_epilogue<kF16, kTileN>(prev, tmem, warp, lane);
        epi_ok = epi_ok && ok;
    }
    failed = __syncthreads_or(failed || !epi_ok) != 0;
    // every MMA this CTA issued has completed before its tensor memory is freed
    // (bounded wait; on a normal exit the last epilogue has already seen them)
    if (tid == 0) {
        mma_commit(bar(5));
        if (!mbar_wait(bar(5), 0u)) failed = true;
    }
    if (failed && tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::kTmemCols));
    }
}

// Operands of the tensor-core forms in one launch (layouts in synth_ops.cuh):
// blocks [0, nbw) compute the weights, one warp per frequency (the FP16 scale
// is that warp's maximum); the other blocks compute the element delays, one
// thread per path and group of kPrepG elements (per transmit element and
// group of kPrepG receive elements for the LoS delays), the reference
// distance once per thread. Blocks of kPrepThreads threads spread the FP64
// work (square roots above all) over every SM.
constexpr int kPrepThreads = 128;
constexpr int kPrepG = 2;
struct TcPrep {
    int32_t Pr, Pp, Nt, Nr, F, nbw;
    const int32_t* nb;       // [Pr] reflections of the receiver's paths
    const double* pts;       // [Pr][kKmax][3]
    const double* L;         // [Pr]
    const float2* g;         // [Pr][F]
    const double* freqs;
    const double* tx_elem;
    const double* rx_elem;
    const double* R0;
    d3 T0;
    float* dtT;              // [Pp/4][Nt][4] (synth_ops.cuh)
    float* drT;              // [Pp/4][Nr][4]
    float* dlos;
    float2* w;
    float2* wl;
    float* sc;
};

__global__ void k_tc_prep(const __grid_constant__ TcPrep a) {
    // the synthesis kernel that follows may start its prologue now (it waits
    // for this grid's results before it reads them)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int n0 = (a.Pr > 0 && a.nb[0] == 0) ? 1 : 0;   // the LoS path sorts first
    const int nrefl = a.Pr - n0;
    if ((int)blockIdx.x < a.nbw) {
        const int f = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
        if (f >= a.F) return;
        const double fr = a.freqs[f];
        float m = 0.f;
        // index Pp is the LoS weight, taken by a lane of the last round (often
        // an idle one) instead of after the reduction
        for (int n = lane; n <= a.Pp; n += 32) {
            if (n == a.Pp) {
                a.wl[f] = n0 ? synth_weight(a.g[f], fr, a.L[0]) : make_float2(0.f, 0.f);
                continue;
            }
            float2 ww = make_float2(0.f, 0.f);
            if (n < nrefl) ww = synth_weight(a.g[(int64_t)(n + n0) * a.F + f], fr, a.L[n + n0]);
            a.w[(int64_t)f * a.Pp + n] = ww;
            m = fmaxf(m, fmaxf(fabsf(ww.x), fabsf(ww.y)));
        }
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) a.sc[f] = synth_scale(m);
        return;
    }
    // delays; consecutive threads write consecutive words of a row
    const int64_t gt = (a.Nt + kPrepG - 1) / kPrepG, gr = (a.Nr + kPrepG - 1) / kPrepG;
    const int64_t n_dt = (int64_t)a.Pp * gt, n_dr = (int64_t)a.Pp * gr, n_dl = (int64_t)a.Nt * gr;
    const int64_t total = n_dt + n_dr + n_dl;
    const int64_t stride = (int64_t)(gridDim.x - a.nbw) * blockDim.x;
    for (int64_t t = (int64_t)(blockIdx.x - a.nbw) * blockDim.x + threadIdx.x; t < total; t += stride) {
        if (t < n_dr + n_dt) {
            const bool tx = t < n_dt;
            const int64_t u = tx ? t : t - n_dt;
            const int n = (int)(u % a.Pp), e0 = (int)(u / a.Pp) * kPrepG;
            const int ne = tx ? a.Nt : a.Nr;
            const double* elem = tx ? a.tx_elem : a.rx_elem;
            // element e, path n at [n / 4][e][n % 4]
            float* dst = (tx ? a.dtT : a.drT) + (int64_t)(n >> 2) * ne * 4 + (n & 3);
            if (n < nrefl) {
                const int i = n + n0, m = a.nb[i];
                const d3 P = ld3(a.pts + ((int64_t)i * kKmax + (tx ? 0 : m - 1)) * 3);
                const double ref = dist_rn(tx ? a.T0 : ld3(a.R0), P);
#pragma unroll
                for (int k = 0; k < kPrepG; ++k)
                    if (e0 + k < ne) dst[(int64_t)(e0 + k) * 4] = el_delay(elem + 3 * (e0 + k), P, ref);
            } else {
#pragma unroll
                for (int k = 0; k < kPrepG; ++k)
                    if (e0 + k < ne) dst[(int64_t)(e0 + k) * 4] = 0.f;
            }
        } else {
            const int64_t u = t - n_dt - n_dr;
            const int p = (int)(u % a.Nt), q0 = (int)(u / a.Nt) * kPrepG;
            const double ref = dist_rn(a.T0, ld3(a.R0));
#pragma unroll
            for (int k = 0; k < kPrepG; ++k)
                if (q0 + k < a.Nr)
                    a.dlos[(int64_t)(q0 + k) * a.Nt + p] = el_delay(a.tx_elem + 3 * p, ld3(a.rx_elem + 3 * (q0 + k)), ref);
        }
    }
}

inline unsigned blocks_of(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, (n + threads - 1) / threads);
}

}  // namespace

sbr_status synth_tc_run(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                        const double* tx_elem, int32_t Nt, const double* rx_elem, int32_t Nr,
                        int32_t rx_index, float2* H, bool f16, cudaStream_t s) {
    const int32_t o0 = pl->h_rx_off[rx_index], Pr = pl->h_rx_off[rx_index + 1] - o0;
    const int32_t Pp = (int32_t)std::max<int64_t>(8, (Pr + 7) & ~7);   // reflected paths, padded
    // one buffer for every operand, 16-byte aligned parts: w, wl (8-byte
    // elements) first, then sc, dtT, drT, dlos
    const size_t n_w = (size_t)Pp * F, n_wl = ((size_t)F + 1) & ~(size_t)1;
    const size_t n_sc = ((size_t)F + 3) & ~(size_t)3;
    const size_t n_f = n_sc + (size_t)Pp * Nt + (size_t)Pp * Nr + (((size_t)Nr * Nt + 3) & ~(size_t)3);
    float2* w;
    SBR_TRY(dalloc_n(&w, n_w + n_wl + (n_f + 1) / 2, s));
    float2* wl = w + n_w;
    float* sc = reinterpret_cast<float*>(wl + n_wl);
    float* dtT = sc + n_sc;
    float* drT = dtT + (size_t)Pp * Nt;
    float* dl = drT + (size_t)Pp * Nr;
    TcPrep pp{};
    pp.Pr = Pr; pp.Pp = Pp; pp.Nt = Nt; pp.Nr = Nr; pp.F = F;
    pp.nb = pl->nb + o0;
    pp.pts = pl->pts + (int64_t)o0 * kKmax * 3;
    pp.L = pl->L + o0;
    pp.g = g + (int64_t)o0 * F;
    pp.freqs = freqs; pp.tx_elem = tx_elem; pp.rx_elem = rx_elem;
    pp.R0 = pl->rx_xyz + 3 * rx_index;
    pp.T0 = mk3(pl->tx[0], pl->tx[1], pl->tx[2]);
    pp.dtT = dtT; pp.drT = drT; pp.dlos = dl; pp.w = w; pp.wl = wl; pp.sc = sc;
    pp.nbw = (int)blocks_of((int64_t)F * 32, kPrepThreads);
    const int64_t gt = (Nt + kPrepG - 1) / kPrepG, gr = (Nr + kPrepG - 1) / kPrepG;
    const int64_t n_del = (int64_t)Pp * (gt + gr) + (int64_t)Nt * gr;
    const unsigned nbd = (unsigned)std::min<int64_t>(blocks_of(n_del, kPrepThreads), 32 * (int64_t)sm_count());
    ::sbr::note_launch(), k_tc_prep<<<(unsigned)pp.nbw + nbd, kPrepThreads, 0, s>>>(pp);
    SBR_TRY_CUDA(cudaGetLastError());
    TcArgs a{};
    a.F = F; a.Nr = Nr; a.Nt = Nt;
    a.Pr = Pr; a.Pp = Pp;
    a.nb0 = pl->nb + o0;
    a.freqs = freqs; a.dtT = dtT; a.drT = drT; a.w = w; a.wl = wl; a.sc = sc; a.dlos = dl; a.H = H;
    a.status = pl->d_status;  // a bounded wait that gave up is reported by sbr_path_query
    a.inject_timeout = fault_mode() == kFaultTimeout ? 1 : 0;
    auto kern = f16 ? k_synth_tc<true, false, 256> : k_synth_tc<false, false, 256>;
    constexpr int kSmemBytes = TcShape<256>::kSmemBytes;
    SBR_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    int64_t items = (int64_t)F * ((Nr + 63) / 64) * ((Nt + 255) / 256);
    // one persistent CTA per SM (two operand stages and two accumulators each),
    // launched as a programmatic dependent of the prologue
    const int grid = (int)std::min<int64_t>(items, (int64_t)sm_count());
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ::sbr::note_launch();
    SBR_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
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
    a.wl_all = w.wl;
    a.sc_all = w.sc;
    a.status = w.status;
    a.inject_timeout = fault_mode() == kFaultTimeout ? 1 : 0;
    if (w.items <= 0) return SBR_OK;
    int grid = (int)std::min<int64_t>(w.items, (int64_t)sm_count());
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
