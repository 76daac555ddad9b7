// Learned surrogate of the channel statistics: a BF16 MLP on Fourier features
// of (x, y, z, f) trained on SBR-traced receivers, with full SBR as fallback.
// The paper has no such model; it is a query-time stand-in for the method's
// outputs (path loss, RMS delay spread, PDP; Eq. 2, 4, 5) learned from them.
//
// Network: 4 inputs -> 128 Fourier features -> depth x width ReLU layers ->
// 128 linear outputs (the first n_out used). Every layer is a GEMM on the
// tcgen05 tensor cores (BF16 operands staged in 128-byte-swizzled shared
// memory, FP32 accumulator in tensor memory) with the bias, ReLU, ReLU-mask
// or atomic split-K reduction fused into the epilogue. Training: mean squared
// error over the finite targets with per-output weights, an optional error
// head learning |prediction - target| of one output (stop-gradient), Adam on
// FP32 master weights with BF16 working copies.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "sbr_internal.cuh"
#include "tcgen05.cuh"

struct sbr_mlp;

namespace sbr {
namespace {
using namespace tc;
using bf16 = __nv_bfloat16;

constexpr int kGThreads = 256;
constexpr int kFeat = 128;      // Fourier features: 4 coordinates x 16 octaves x (sin, cos)
constexpr int kOctaves = 16;
constexpr int kOutW = 128;      // output layer width (first n_out used)

enum { kEpReluBf16 = 0, kEpBiasF32 = 1, kEpMaskBf16 = 2, kEpAtomicF32 = 3 };

struct GemmArgs {
    const bf16* A;        // [M][K], K contiguous
    const bf16* B;        // [N][K]
    int M, N, K;          // M % 128 == 0, N % tile == 0, K % 64 == 0
    int k_split;          // K elements per blockIdx.z
    const float* bias;    // [N] (bias epilogues)
    const bf16* mask;     // [M][N] (mask epilogue: keep where mask > 0)
    bf16* Cb;             // [M][N] BF16 out
    float* Cf;            // [M][N] FP32 out
    unsigned int* status;
};

template <int kN>
struct GemmShape {
    static constexpr int kStage = 128 * 128 + kN * 128;   // A and B chunks of 64 BF16 per row
    static constexpr int kSmemTiles = 2 * kStage;          // two stages
    // at least the tiles, and enough that at most 512 / kN CTAs share an SM, so
    // their tensor-memory allocations (kN columns each) always fit
    static constexpr int kTmemReq = 228 * 1024 / (512 / kN + 1) + 1024;
    static constexpr int kSmemReq = kSmemTiles + 1024 + 64 > kTmemReq ? kSmemTiles + 1024 + 64 : kTmemReq;
};

// C = A B^T (FP32 accumulation) with a fused epilogue
template <int kN, int kMode>
__global__ void __launch_bounds__(kGThreads, 1) k_gemm(const __grid_constant__ GemmArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    using Sh = GemmShape<kN>;
    uint64_t* mbar = (uint64_t*)(smem + Sh::kSmemTiles);
    uint32_t* tmem_slot = (uint32_t*)(smem + Sh::kSmemTiles + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar + k)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * kN;
    const int k0 = blockIdx.z * a.k_split, k1 = min(a.K, k0 + a.k_split);
    // 16-byte vectors of 8 BF16 of K-chunk kc into the swizzled K-major tiles of
    // stage b, with cp.async: chunk kc + 1 is in flight while chunk kc's MMAs run
    auto issue = [&](int kc, int b) {
        unsigned char* sA = smem + b * Sh::kStage;
        unsigned char* sB = sA + 128 * 128;
        for (int e = tid; e < 128 * 8; e += kGThreads) {
            int r = e >> 3, v = e & 7;
            cp_async16(smem_u32(sA + r * 128 + ((v ^ (r & 7)) << 4)), a.A + (size_t)(m0 + r) * a.K + kc + 8 * v);
        }
        for (int e = tid; e < kN * 8; e += kGThreads) {
            int r = e >> 3, v = e & 7;
            cp_async16(smem_u32(sB + r * 128 + ((v ^ (r & 7)) << 4)), a.B + (size_t)(n0 + r) * a.K + kc + 8 * v);
        }
        cp_async_commit();
    };
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool failed = false;
    const int nchunks = k1 > k0 ? (k1 - k0 + 63) / 64 : 0;
    if (nchunks > 0) issue(k0, 0);
    for (int i = 0; i < nchunks && !failed; ++i) {
        const int bi = i & 1;
        if (i + 1 < nchunks) {
            const int nb = bi ^ 1;
            if (pending[nb]) {   // the MMAs of chunk i - 1 read stage nb
                const bool ok = mbar_wait(smem_u32(mbar + nb), phase[nb]);
                phase[nb] ^= 1u;
                pending[nb] = false;
                if (__syncthreads_or(!ok)) { failed = true; break; }
            }
            issue(k0 + 64 * (i + 1), nb);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* sA = smem + bi * Sh::kStage;
            uint64_t dA = make_desc(smem_u32(sA)), dB = make_desc(smem_u32(sA + 128 * 128));
            for (int ks = 0; ks < 4; ++ks) {
                uint64_t off = (uint64_t)(ks * 32) >> 4;   // 16 BF16 along K
                mma_16<false, kN>(tmem, dA + off, dB + off, (i > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(mbar + bi));
        }
        pending[bi] = true;
    }
    cp_async_wait<0>();
    for (int b = 0; b < 2 && !failed; ++b) {   // every MMA of the tile has completed after both
        if (!pending[b]) continue;
        const bool ok = mbar_wait(smem_u32(mbar + b), phase[b]);
        if (__syncthreads_or(!ok)) failed = true;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool any = nchunks > 0;
    if (failed && tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    if (any && !failed) {
        const int qw = warp & 3, chalf = warp >> 2;
        const int row = m0 + 32 * qw + lane;
        for (int j = 0; j < kN / 64; ++j) {
            const int col0 = (kN / 2) * chalf + 32 * j;
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)col0, v);
            const int c0 = n0 + col0;
            if (kMode == kEpReluBf16 || kMode == kEpMaskBf16) {
                __align__(16) bf16 o[32];
                for (int k = 0; k < 32; ++k) {
                    float x = __uint_as_float(v[k]);
                    if (kMode == kEpReluBf16) x = fmaxf(x + a.bias[c0 + k], 0.f);
                    else x = __bfloat162float(a.mask[(size_t)row * a.N + c0 + k]) > 0.f ? x : 0.f;
                    o[k] = __float2bfloat16_rn(x);
                }
                uint4* dst = reinterpret_cast<uint4*>(a.Cb + (size_t)row * a.N + c0);
                const uint4* src = reinterpret_cast<const uint4*>(o);
                for (int k = 0; k < 4; ++k) dst[k] = src[k];
            } else if (kMode == kEpBiasF32) {
                float4* dst = reinterpret_cast<float4*>(a.Cf + (size_t)row * a.N + c0);
                for (int k = 0; k < 8; ++k)
                    dst[k] = make_float4(__uint_as_float(v[4 * k]) + a.bias[c0 + 4 * k],
                                         __uint_as_float(v[4 * k + 1]) + a.bias[c0 + 4 * k + 1],
                                         __uint_as_float(v[4 * k + 2]) + a.bias[c0 + 4 * k + 2],
                                         __uint_as_float(v[4 * k + 3]) + a.bias[c0 + 4 * k + 3]);
            } else {
                for (int k = 0; k < 32; ++k) atomicAdd(a.Cf + (size_t)row * a.N + c0 + k, __uint_as_float(v[k]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kN));
}

// Fourier features of x = (x, y, z, f) mapped to u in [0, 1]^4: for coordinate
// c and octave k, sin and cos of pi 2^(k lmax / 15) u_c; rows >= B are zero
__global__ void k_features(const float* __restrict__ x, int B, int Mp, float4 lo, float4 inv, float lmax,
                           bf16* __restrict__ feat) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Mp * 4 * kOctaves) return;
    int b = t / (4 * kOctaves), r = t - b * 4 * kOctaves;
    int c = r / kOctaves, k = r - c * kOctaves;
    float s = 0.f, co = 0.f;
    if (b < B) {
        float xv = x[4 * b + c];
        float lov = c == 0 ? lo.x : (c == 1 ? lo.y : (c == 2 ? lo.z : lo.w));
        float iv = c == 0 ? inv.x : (c == 1 ? inv.y : (c == 2 ? inv.z : inv.w));
        float u = (xv - lov) * iv;
        float w = exp2f(lmax * (float)k / 15.0f);
        sincospif(w * u, &s, &co);
    }
    feat[(size_t)b * kFeat + c * 2 * kOctaves + 2 * k] = __float2bfloat16_rn(s);
    feat[(size_t)b * kFeat + c * 2 * kOctaves + 2 * k + 1] = __float2bfloat16_rn(co);
}

// loss and its gradient with respect to the outputs (BF16, zero where unused):
//   L = (1/B) sum_{b, o finite} w_o (p_bo - y'_bo)^2
//     + (1/B) sum_{b: y_b,c finite} w_e (p_be - |p_bc - y'_bc|)^2   (error head e of output c)
// on the normalised targets y' = (y - shift) / scale; outputs are normalised
// units (the error head in those of output c)
__global__ void k_loss(const float* __restrict__ P, const float* __restrict__ Y, int B, int Mp, int n_out,
                       const float* __restrict__ w, const float* __restrict__ shift, const float* __restrict__ scale,
                       int e_ch, int e_of, bf16* __restrict__ dP, float* __restrict__ loss) {
    __shared__ float red[kGThreads / 32];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (t < Mp * kOutW) {
        int b = t / kOutW, o = t - b * kOutW;
        float g = 0.f;
        if (b < B && o < n_out) {
            float p = P[(size_t)b * kOutW + o];
            if (o == e_ch && e_of >= 0) {
                float yc = (Y[(size_t)b * n_out + e_of] - shift[e_of]) / scale[e_of];
                if (isfinite(yc)) {
                    float tgt = fabsf(P[(size_t)b * kOutW + e_of] - yc);
                    float d = p - tgt;
                    l = w[o] * d * d / B;
                    g = 2.f * w[o] * d / B;
                }
            } else {
                float y = (Y[(size_t)b * n_out + o] - shift[o]) / scale[o];
                if (isfinite(y)) {
                    float d = p - y;
                    l = w[o] * d * d / B;
                    g = 2.f * w[o] * d / B;
                }
            }
        }
        dP[t] = __float2bfloat16_rn(g);
    }
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        float s = 0.f;
        for (int k = 0; k < kGThreads / 32; ++k) s += red[k];
        atomicAdd(loss, s);
    }
}

// out[c][r] = in[r][c] for a [R][C] BF16 matrix (32 x 32 tiles through shared memory)
__global__ void k_transpose(const bf16* __restrict__ in, int R, int C, bf16* __restrict__ out) {
    __shared__ bf16 tile[32][33];
    int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int r = r0 + k;
        tile[k][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    int r = r0 + threadIdx.x;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int cc = blockIdx.x * 32 + k;
        if (cc < C && r < R) out[(size_t)cc * R + r] = tile[threadIdx.x][k];
    }
}

// db[n] += sum over rows of d[row][n]
__global__ void k_colsum(const bf16* __restrict__ d, int M, int N, float* __restrict__ db) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int r0 = blockIdx.y * 256, r1 = min(M, r0 + 256);
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += __bfloat162float(d[(size_t)r * N + n]);
    atomicAdd(db + n, s);
}

// Adam on FP32 masters; refreshes the BF16 copy (and its transpose for weights)
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t n, int cols, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16* __restrict__ pb, bf16* __restrict__ pt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
    if (pt) {
        int64_t r = i / cols, c = i - r * cols;
        pt[c * (n / cols) + r] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float* __restrict__ p, int64_t n, int cols, bf16* __restrict__ pb,
                          bf16* __restrict__ pt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pb[i] = __float2bfloat16_rn(p[i]);
    if (pt) {
        int64_t r = i / cols, c = i - r * cols;
        pt[c * (n / cols) + r] = pb[i];
    }
}

// outputs back to target units: y = p scale + shift
__global__ void k_take_outputs(const float* __restrict__ P, int B, int n_out, const float* __restrict__ shift,
                               const float* __restrict__ scale, float* __restrict__ y) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * n_out) return;
    int b = t / n_out, o = t - b * n_out;
    y[t] = P[(size_t)b * kOutW + o] * scale[o] + shift[o];
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ---------------------------------------------------------------- fused inference
// The whole network for 128 rows per tile in one CTA. The features are written
// straight into a shared-memory activation tile; each layer's MMAs read it, and
// its bias + ReLU epilogue (run after those MMAs have completed) overwrites it
// in place with the next layer's BF16 activations, in the MMA's own swizzled
// layout. The weight K-chunks (a fixed sequence per tile) stream from L2 through
// a ring of kStages shared-memory stages with cp.async, kStages - 1 chunks
// ahead of the MMAs and across layer and tile boundaries; the accumulator is in
// TMEM. Only the inputs and the n_out outputs touch HBM.
constexpr int kMaxLayers = 9;
constexpr int kStages = 4;
constexpr int kActBytes = 128 * 256 * 2;    // 128 rows x 256 BF16, four 16 KB K-chunk tiles
constexpr int kBChunkBytes = 256 * 128;     // up to 256 weight rows x 64 BF16
constexpr int kInferSmem = kActBytes + kStages * kBChunkBytes + 1024 + 128;

struct InferArgs {
    const float* x;
    int B;
    float4 lo, inv;
    float lmax;
    int n_layers;
    const bf16* W[kMaxLayers];
    const float* bias[kMaxLayers];
    int n_in[kMaxLayers];
    int n_out[kMaxLayers];
    int n_used;
    const float* shift;
    const float* scale;
    float* y;
    unsigned int* status;
};

__device__ __forceinline__ uint32_t act_off(int r, int k) {   // byte offset in the activation tile
    return (uint32_t)(k >> 6) * (128 * 128) + sw128(r, k & 63);
}

__global__ void __launch_bounds__(kGThreads, 1) k_mlp_infer(const __grid_constant__ InferArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* act = smem;
    unsigned char* ring = smem + kActBytes;
    uint64_t* mbar = (uint64_t*)(smem + kActBytes + kStages * kBChunkBytes);
    uint32_t* tmem_slot = (uint32_t*)(mbar + kStages);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < kStages; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar + k)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // the per-tile chunk sequence: layer l has n_in[l] / 64 chunks
    int per_tile = 0;
    for (int l = 0; l < a.n_layers; ++l) per_tile += a.n_in[l] / 64;
    const int ntiles = (a.B + 127) / 128;
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = (int64_t)my_tiles * per_tile;   // chunks this CTA consumes
    // copy of chunk g (of this CTA's sequence) into its stage
    auto issue = [&](int64_t g) {
        if (g < total) {
            int q = (int)(g % per_tile), l = 0;
            while (q >= a.n_in[l] / 64) { q -= a.n_in[l] / 64; ++l; }
            const int K = a.n_in[l], N = a.n_out[l];
            const bf16* W = a.W[l];
            unsigned char* st = ring + (int)(g % kStages) * kBChunkBytes;
            for (int e = tid; e < N * 8; e += kGThreads) {
                int r = e >> 3, v = e & 7;
                cp_async16(smem_u32(st + r * 128 + ((v ^ (r & 7)) << 4)), W + (size_t)r * K + q * 64 + 8 * v);
            }
        }
        cp_async_commit();   // one group per chunk, empty past the end, so the group count stays fixed
    };
    uint32_t phase_bits = 0u;   // parity to wait for, per stage
    bool failed = false;
    // consume the MMA commits of chunks up to c, each exactly once and in order
    // (a stage's barrier completes once per chunk that used it)
    int64_t waited = -1;
    auto wait_chunk = [&](int64_t c) -> bool {
        while (waited < c) {
            ++waited;
            const int sp = (int)(waited % kStages);
            // at most 2^21 tries of up to 1 us: a wait that never ends gives up within seconds
            const bool ok = mbar_wait_sleep(smem_u32(mbar + sp), (phase_bits >> sp) & 1u, 1000u, 1u << 21);
            phase_bits ^= 1u << sp;
            if (__syncthreads_or(!ok)) return false;
        }
        return true;
    };
    for (int64_t c = 0; c < kStages - 1; ++c) issue(c);
    int64_t g = 0;              // next chunk to consume
    const int qw = warp & 3, chalf = warp >> 2;
    for (int t = 0; t < my_tiles && !failed; ++t) {
        const int r0 = (blockIdx.x + t * gridDim.x) * 128;
        // Fourier features of the tile's rows (the previous tile's MMAs have completed)
        for (int e = tid; e < 128 * 4 * kOctaves; e += kGThreads) {
            int r = e / (4 * kOctaves), q = e - r * 4 * kOctaves;
            int c = q / kOctaves, k = q - c * kOctaves;
            float s = 0.f, co = 0.f;
            if (r0 + r < a.B) {
                float xv = a.x[4 * (r0 + r) + c];
                float lov = c == 0 ? a.lo.x : (c == 1 ? a.lo.y : (c == 2 ? a.lo.z : a.lo.w));
                float iv = c == 0 ? a.inv.x : (c == 1 ? a.inv.y : (c == 2 ? a.inv.z : a.inv.w));
                sincospif(exp2f(a.lmax * (float)k / 15.0f) * ((xv - lov) * iv), &s, &co);
            }
            const int f = c * 2 * kOctaves + 2 * k;
            *reinterpret_cast<__nv_bfloat162*>(act + act_off(r, f)) = __floats2bfloat162_rn(s, co);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int l = 0; l < a.n_layers && !failed; ++l) {
            const int N = a.n_out[l], nch = a.n_in[l] / 64;
            for (int kc = 0; kc < nch; ++kc, ++g) {
                // chunks up to g + kStages - 2 are issued: all but the newest
                // kStages - 2 groups complete means chunk g has landed
                cp_async_wait<kStages - 2>();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int sg = (int)(g % kStages);
                    uint64_t dA = make_desc(smem_u32(act + kc * (128 * 128)));
                    uint64_t dB = make_desc(smem_u32(ring + sg * kBChunkBytes));
                    for (int ks = 0; ks < 4; ++ks) {
                        uint64_t off = (uint64_t)(ks * 32) >> 4;
                        uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                        if (N == 256) mma_16<false, 256>(tmem, dA + off, dB + off, acc);
                        else mma_16<false, 128>(tmem, dA + off, dB + off, acc);
                    }
                    mma_commit(smem_u32(mbar + sg));
                }
                // with chunk g's MMAs queued, recycle the stage of chunk g - 1 (its
                // MMAs precede g's) for chunk g + kStages - 1
                if (!wait_chunk(g - 1)) { failed = true; break; }
                issue(g + kStages - 1);
            }
            if (failed) break;
            // every MMA of the layer has completed once its last chunk's commit has
            if (!wait_chunk(g - 1)) { failed = true; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = 32 * qw + lane;
            const bool last = l + 1 == a.n_layers;
            for (int j = 0; j < N / 64; ++j) {
                const int col0 = (N / 2) * chalf + 32 * j;
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)col0, v);
                if (!last) {
                    for (int k = 0; k < 32; k += 8) {
                        __align__(16) __nv_bfloat162 o[4];
                        for (int u = 0; u < 4; ++u) {
                            float x0 = fmaxf(__uint_as_float(v[k + 2 * u]) + a.bias[l][col0 + k + 2 * u], 0.f);
                            float x1 = fmaxf(__uint_as_float(v[k + 2 * u + 1]) + a.bias[l][col0 + k + 2 * u + 1], 0.f);
                            o[u] = __floats2bfloat162_rn(x0, x1);
                        }
                        *reinterpret_cast<uint4*>(act + act_off(row, col0 + k)) = *reinterpret_cast<uint4*>(o);
                    }
                } else if (r0 + row < a.B) {
                    for (int k = 0; k < 32; ++k) {
                        const int o = col0 + k;
                        if (o < a.n_used)
                            a.y[(size_t)(r0 + row) * a.n_used + o] =
                                (__uint_as_float(v[k]) + a.bias[l][o]) * a.scale[o] + a.shift[o];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
    }
    cp_async_wait<0>();
    if (failed && tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

template <int kN, int kMode>
sbr_status gemm_launch(const GemmArgs& a, int splits, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    SBR_TRY(set_smem_once((const void*)k_gemm<kN, kMode>, GemmShape<kN>::kSmemReq, &attr));
    dim3 grid(a.M / 128, a.N / kN, splits);
    ::sbr::note_launch(), k_gemm<kN, kMode><<<grid, kGThreads, GemmShape<kN>::kSmemReq, s>>>(a);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

// dispatch on the tile width (the whole N when it is 128 or 256)
template <int kMode>
sbr_status gemm(const GemmArgs& a, int splits, cudaStream_t s) {
    if (a.M % 128 || a.K % 64 || a.K <= 0) { set_error("gemm shape M=%d K=%d", a.M, a.K); return SBR_ERR_INVALID_ARG; }
    if (a.N % 256 == 0) return gemm_launch<256, kMode>(a, splits, s);
    if (a.N % 128 == 0) return gemm_launch<128, kMode>(a, splits, s);
    set_error("gemm N=%d not a multiple of 128", a.N);
    return SBR_ERR_INVALID_ARG;
}

struct Layer {
    int n_in, n_out;
    float* W = nullptr;      // [n_out][n_in] FP32 master
    float* b = nullptr;      // [n_out]
    float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
    float* gW = nullptr;     // gradients
    float* gb = nullptr;
    bf16* Wb = nullptr;      // BF16 [n_out][n_in]
    bf16* Wt = nullptr;      // BF16 [n_in][n_out]
    bf16* H = nullptr;       // activation out [Mp][n_out] (hidden layers)
    bf16* Ht = nullptr;      // its transpose [n_out][Mp]
    bf16* dH = nullptr;      // gradient w.r.t. the output [Mp][n_out]
    bf16* dHt = nullptr;     // its transpose
};

}  // namespace
}  // namespace sbr

struct sbr_mlp {
    int device = 0;
    sbr_mlp_config cfg{};
    int Mp = 0;                        // max_batch rounded up to 128
    std::vector<sbr::Layer> L;         // depth hidden + output
    std::vector<float> loss_w;         // [n_out]
    float* d_loss_w = nullptr;         // [128] loss weights
    float* d_shift = nullptr;          // [128] target normalisation
    float* d_scale = nullptr;
    sbr::bf16* feat = nullptr;         // [Mp][128]
    sbr::bf16* featT = nullptr;        // [128][Mp]
    float* P = nullptr;                // [Mp][128] outputs
    unsigned int* status = nullptr;
    int64_t step = 0;
    std::vector<void*> owned;
};

namespace sbr {
namespace {

template <class T>
sbr_status malloc_owned(sbr_mlp* m, T** p, size_t n) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("mlp allocation of %zu bytes: %s", n * sizeof(T), cudaGetErrorString(e));
        return SBR_ERR_ALLOC;
    }
    m->owned.push_back(*p);
    return SBR_OK;
}

void free_mlp(sbr_mlp* m) {
    if (!m) return;
    cudaDeviceSynchronize();
    for (void* p : m->owned) cudaFree(p);
    delete m;
}

// splitmix64: seeded, platform-independent initial weights
uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

sbr_status forward(const sbr_mlp* m, const float* x, int B, cudaStream_t s) {
    const sbr_mlp_config& c = m->cfg;
    const int Mp = ((B + 127) / 128) * 128;
    float4 lo = make_float4(c.x_lo[0], c.x_lo[1], c.x_lo[2], c.x_lo[3]);
    float4 inv = make_float4(1.f / (c.x_hi[0] - c.x_lo[0]), 1.f / (c.x_hi[1] - c.x_lo[1]),
                             1.f / (c.x_hi[2] - c.x_lo[2]), 1.f / (c.x_hi[3] - c.x_lo[3]));
    ::sbr::note_launch(), k_features<<<nblk((int64_t)Mp * 4 * kOctaves), 256, 0, s>>>(x, B, Mp, lo, inv,
                                                                                      c.feat_log2_max, m->feat);
    SBR_TRY_CUDA(cudaGetLastError());
    const bf16* in = m->feat;
    for (size_t l = 0; l < m->L.size(); ++l) {
        const Layer& ly = m->L[l];
        GemmArgs a{};
        a.A = in;
        a.B = ly.Wb;
        a.M = Mp;
        a.N = ly.n_out;
        a.K = ly.n_in;
        a.k_split = ly.n_in;
        a.bias = ly.b;
        a.status = m->status;
        if (l + 1 < m->L.size()) {
            a.Cb = ly.H;
            SBR_TRY(gemm<kEpReluBf16>(a, 1, s));
            in = ly.H;
        } else {
            a.Cf = m->P;
            SBR_TRY(gemm<kEpBiasF32>(a, 1, s));
        }
    }
    return SBR_OK;
}

sbr_status transpose(const bf16* in, int R, int C, bf16* out, cudaStream_t s) {
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    ::sbr::note_launch(), k_transpose<<<grid, block, 0, s>>>(in, R, C, out);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

sbr_status train_step(sbr_mlp* m, const float* x, const float* y, int B, float* loss, cudaStream_t s) {
    const sbr_mlp_config& c = m->cfg;
    const int Mp = ((B + 127) / 128) * 128;
    SBR_TRY(forward(m, x, B, s));
    const int nl = (int)m->L.size();
    Layer& out = m->L[nl - 1];
    ::sbr::note_launch(), k_loss<<<nblk((int64_t)Mp * kOutW), kGThreads, 0, s>>>(
        m->P, y, B, Mp, c.n_out, m->d_loss_w, m->d_shift, m->d_scale, c.err_channel, c.err_of, out.dH, loss);
    SBR_TRY_CUDA(cudaGetLastError());
    // backward: for each layer, dW = dH^T X (split-K atomics), db = column sums,
    // then the input gradient (dH W) masked by the previous ReLU
    for (int l = nl - 1; l >= 0; --l) {
        Layer& ly = m->L[l];
        const bf16* X = l > 0 ? m->L[l - 1].H : m->feat;
        bf16* Xt = l > 0 ? m->L[l - 1].Ht : m->featT;
        SBR_TRY_CUDA(cudaMemsetAsync(ly.gW, 0, sizeof(float) * (size_t)ly.n_out * ly.n_in, s));
        SBR_TRY_CUDA(cudaMemsetAsync(ly.gb, 0, sizeof(float) * ly.n_out, s));
        SBR_TRY(transpose(ly.dH, Mp, ly.n_out, ly.dHt, s));
        SBR_TRY(transpose(X, Mp, ly.n_in, Xt, s));
        GemmArgs gw{};
        gw.A = ly.dHt;
        gw.B = Xt;
        gw.M = ly.n_out;
        gw.N = ly.n_in;
        gw.K = Mp;
        const int splits = std::max(1, std::min(Mp / 512, 32));
        gw.k_split = ((Mp / splits + 63) / 64) * 64;
        gw.Cf = ly.gW;
        gw.status = m->status;
        SBR_TRY(gemm<kEpAtomicF32>(gw, (Mp + gw.k_split - 1) / gw.k_split, s));
        dim3 cg(nblk(ly.n_out), (Mp + 255) / 256);
        ::sbr::note_launch(), k_colsum<<<cg, 256, 0, s>>>(ly.dH, Mp, ly.n_out, ly.gb);
        SBR_TRY_CUDA(cudaGetLastError());
        if (l > 0) {
            GemmArgs gx{};
            gx.A = ly.dH;
            gx.B = ly.Wt;
            gx.M = Mp;
            gx.N = ly.n_in;
            gx.K = ly.n_out;
            gx.k_split = ly.n_out;
            gx.mask = m->L[l - 1].H;
            gx.Cb = m->L[l - 1].dH;
            gx.status = m->status;
            SBR_TRY(gemm<kEpMaskBf16>(gx, 1, s));
        }
    }
    m->step += 1;
    const float c1 = 1.f - powf(c.beta1, (float)m->step), c2 = 1.f - powf(c.beta2, (float)m->step);
    for (Layer& ly : m->L) {
        const int64_t nw = (int64_t)ly.n_out * ly.n_in;
        ::sbr::note_launch(), k_adam<<<nblk(nw), 256, 0, s>>>(ly.W, ly.mW, ly.vW, ly.gW, nw, ly.n_in, c.lr, c.beta1,
                                                              c.beta2, c.eps, c1, c2, ly.Wb, ly.Wt);
        ::sbr::note_launch(), k_adam<<<nblk(ly.n_out), 256, 0, s>>>(ly.b, ly.mb, ly.vb, ly.gb, ly.n_out, 1, c.lr,
                                                                    c.beta1, c.beta2, c.eps, c1, c2, nullptr, nullptr);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    return SBR_OK;
}

sbr_status sync_bf16(sbr_mlp* m, cudaStream_t s) {
    for (Layer& ly : m->L) {
        const int64_t nw = (int64_t)ly.n_out * ly.n_in;
        ::sbr::note_launch(), k_to_bf16<<<nblk(nw), 256, 0, s>>>(ly.W, nw, ly.n_in, ly.Wb, ly.Wt);
        SBR_TRY_CUDA(cudaGetLastError());
    }
    return SBR_OK;
}

sbr_status infer_fused(const sbr_mlp* m, const float* x, int B, float* y, cudaStream_t s) {
    const sbr_mlp_config& c = m->cfg;
    static std::atomic<unsigned long long> attr{0};
    SBR_TRY(set_smem_once((const void*)k_mlp_infer, kInferSmem, &attr));
    InferArgs a{};
    a.x = x;
    a.B = B;
    a.lo = make_float4(c.x_lo[0], c.x_lo[1], c.x_lo[2], c.x_lo[3]);
    a.inv = make_float4(1.f / (c.x_hi[0] - c.x_lo[0]), 1.f / (c.x_hi[1] - c.x_lo[1]),
                        1.f / (c.x_hi[2] - c.x_lo[2]), 1.f / (c.x_hi[3] - c.x_lo[3]));
    a.lmax = c.feat_log2_max;
    a.n_layers = (int)m->L.size();
    for (int l = 0; l < a.n_layers; ++l) {
        a.W[l] = m->L[l].Wb;
        a.bias[l] = m->L[l].b;
        a.n_in[l] = m->L[l].n_in;
        a.n_out[l] = m->L[l].n_out;
    }
    a.n_used = c.n_out;
    a.shift = m->d_shift;
    a.scale = m->d_scale;
    a.y = y;
    a.status = m->status;
    const int ntiles = (B + 127) / 128;
    const int grid = std::min(ntiles, sm_count());
    ::sbr::note_launch(), k_mlp_infer<<<grid, kGThreads, kInferSmem, s>>>(a);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

int64_t n_params(const sbr_mlp* m) {
    int64_t n = 0;
    for (const Layer& ly : m->L) n += (int64_t)ly.n_out * ly.n_in + ly.n_out;
    return n;
}

}  // namespace
}  // namespace sbr

using namespace sbr;

extern "C" {

sbr_status sbr_mlp_create(const sbr_mlp_config* cfg, const float* loss_w, const float* y_shift,
                          const float* y_scale, sbr_mlp** out, void* stream) {
    clear_error();
    SBR_CHECK_ARG(cfg && out, "config and out");
    *out = nullptr;
    const sbr_mlp_config& c = *cfg;
    SBR_CHECK_ARG(c.n_out >= 1 && c.n_out <= kOutW, "n_out in [1, 128]");
    SBR_CHECK_ARG(c.width == 128 || c.width == 256, "width 128 or 256");
    SBR_CHECK_ARG(c.depth >= 1 && c.depth <= 8, "depth in [1, 8]");
    SBR_CHECK_ARG(c.max_batch >= 1 && c.max_batch <= (1 << 22), "max_batch in [1, 2^22]");
    SBR_CHECK_ARG((c.err_of < 0 && c.err_channel < 0) ||
                      (c.err_of >= 0 && c.err_channel >= 0 && c.err_of < c.n_out && c.err_channel < c.n_out &&
                       c.err_of != c.err_channel),
                  "error head channels: both -1, or two different outputs");
    for (int k = 0; k < 4; ++k) SBR_CHECK_ARG(c.x_hi[k] > c.x_lo[k], "x_hi > x_lo");
    SBR_CHECK_ARG(c.feat_log2_max >= 0.f && c.feat_log2_max <= 20.f, "feat_log2_max in [0, 20]");
    SBR_CHECK_ARG(c.lr > 0.f && c.beta1 >= 0.f && c.beta1 < 1.f && c.beta2 >= 0.f && c.beta2 < 1.f && c.eps > 0.f,
                  "Adam hyper-parameters");
    sbr_mlp* m = new (std::nothrow) sbr_mlp();
    if (!m) { set_error("host allocation"); return SBR_ERR_ALLOC; }
    SBR_TRY_CUDA(cudaGetDevice(&m->device));
    m->cfg = c;
    if (m->cfg.feat_log2_max == 0.f) m->cfg.feat_log2_max = 9.f;
    m->Mp = ((c.max_batch + 127) / 128) * 128;
    m->loss_w.assign(c.n_out, 1.f);
    if (loss_w) for (int k = 0; k < c.n_out; ++k) m->loss_w[k] = loss_w[k];
    auto fail = [&](sbr_status st) { free_mlp(m); return st; };
    sbr_status st;
    const int Mp = m->Mp;
    std::vector<int> widths;
    widths.push_back(kFeat);
    for (int d = 0; d < c.depth; ++d) widths.push_back(c.width);
    widths.push_back(kOutW);
    uint64_t rs = c.seed;
    std::vector<float> host;
    for (size_t l = 0; l + 1 < widths.size(); ++l) {
        Layer ly;
        ly.n_in = widths[l];
        ly.n_out = widths[l + 1];
        const size_t nw = (size_t)ly.n_in * ly.n_out;
        if ((st = malloc_owned(m, &ly.W, nw)) || (st = malloc_owned(m, &ly.b, ly.n_out)) ||
            (st = malloc_owned(m, &ly.mW, nw)) || (st = malloc_owned(m, &ly.vW, nw)) ||
            (st = malloc_owned(m, &ly.mb, ly.n_out)) || (st = malloc_owned(m, &ly.vb, ly.n_out)) ||
            (st = malloc_owned(m, &ly.gW, nw)) || (st = malloc_owned(m, &ly.gb, ly.n_out)) ||
            (st = malloc_owned(m, &ly.Wb, nw)) || (st = malloc_owned(m, &ly.Wt, nw)) ||
            (st = malloc_owned(m, &ly.H, (size_t)Mp * ly.n_out)) || (st = malloc_owned(m, &ly.Ht, (size_t)Mp * ly.n_out)) ||
            (st = malloc_owned(m, &ly.dH, (size_t)Mp * ly.n_out)) || (st = malloc_owned(m, &ly.dHt, (size_t)Mp * ly.n_out)))
            return fail(st);
        // He-uniform weights, zero biases
        host.resize(nw);
        const float lim = std::sqrt(6.0f / (float)ly.n_in) * (l + 2 == widths.size() ? 0.1f : 1.0f);
        for (size_t i = 0; i < nw; ++i) host[i] = lim * (2.0f * (float)((splitmix(rs) >> 40) * (1.0 / 16777216.0)) - 1.0f);
        if (cudaMemcpy(ly.W, host.data(), nw * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(ly.b, 0, ly.n_out * 4) != cudaSuccess || cudaMemset(ly.mW, 0, nw * 4) != cudaSuccess ||
            cudaMemset(ly.vW, 0, nw * 4) != cudaSuccess || cudaMemset(ly.mb, 0, ly.n_out * 4) != cudaSuccess ||
            cudaMemset(ly.vb, 0, ly.n_out * 4) != cudaSuccess) {
            set_error("mlp initialisation copy failed");
            return fail(SBR_ERR_CUDA);
        }
        m->L.push_back(ly);
    }
    if ((st = malloc_owned(m, &m->feat, (size_t)Mp * kFeat)) || (st = malloc_owned(m, &m->featT, (size_t)Mp * kFeat)) ||
        (st = malloc_owned(m, &m->P, (size_t)Mp * kOutW)) || (st = malloc_owned(m, &m->status, 1)) ||
        (st = malloc_owned(m, &m->d_loss_w, kOutW)) || (st = malloc_owned(m, &m->d_shift, kOutW)) ||
        (st = malloc_owned(m, &m->d_scale, kOutW)))
        return fail(st);
    std::vector<float> lw(kOutW, 0.f), sh(kOutW, 0.f), sc(kOutW, 1.f);
    for (int k = 0; k < c.n_out; ++k) {
        lw[k] = m->loss_w[k];
        if (y_shift) sh[k] = y_shift[k];
        if (y_scale) sc[k] = y_scale[k];
        if (!(sc[k] > 0.f) || !std::isfinite(sh[k])) {
            set_error("y_scale must be > 0 and y_shift finite (output %d)", k);
            return fail(SBR_ERR_INVALID_ARG);
        }
    }
    if (cudaMemcpy(m->d_loss_w, lw.data(), kOutW * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->d_shift, sh.data(), kOutW * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->d_scale, sc.data(), kOutW * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->status, 0, 4) != cudaSuccess) {
        set_error("mlp initialisation copy failed");
        return fail(SBR_ERR_CUDA);
    }
    if ((st = sync_bf16(m, (cudaStream_t)stream)) != SBR_OK) return fail(st);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return fail(SBR_ERR_CUDA);
    *out = m;
    return SBR_OK;
}

sbr_status sbr_mlp_train_step(sbr_mlp* m, const float* x, const float* y, int32_t B, float* loss, void* stream) {
    clear_error();
    SBR_CHECK_ARG(m && x && y, "mlp, x, y");
    SBR_CHECK_ARG(B >= 1 && B <= m->cfg.max_batch, "1 <= B <= max_batch");
    return train_step(m, x, y, B, loss, (cudaStream_t)stream);
}

sbr_status sbr_mlp_predict(const sbr_mlp* m, const float* x, int32_t B, float* y, void* stream) {
    clear_error();
    SBR_CHECK_ARG(m && x && y, "mlp, x, y");
    SBR_CHECK_ARG(B >= 1 && B <= m->cfg.max_batch, "1 <= B <= max_batch");
    cudaStream_t s = (cudaStream_t)stream;
    return infer_fused(m, x, B, y, s);
}

sbr_status sbr_mlp_predict_layered(const sbr_mlp* m, const float* x, int32_t B, float* y, void* stream) {
    clear_error();
    SBR_CHECK_ARG(m && x && y, "mlp, x, y");
    SBR_CHECK_ARG(B >= 1 && B <= m->cfg.max_batch, "1 <= B <= max_batch");
    cudaStream_t s = (cudaStream_t)stream;
    SBR_TRY(forward(m, x, B, s));
    ::sbr::note_launch(), k_take_outputs<<<nblk((int64_t)B * m->cfg.n_out), 256, 0, s>>>(m->P, B, m->cfg.n_out,
                                                                                      m->d_shift, m->d_scale, y);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

int64_t sbr_mlp_param_count(const sbr_mlp* m) { return m ? n_params(m) : 0; }

sbr_status sbr_mlp_params(sbr_mlp* m, float* params, int32_t mode, void* stream) {
    clear_error();
    SBR_CHECK_ARG(m && params, "mlp and params");
    SBR_CHECK_ARG(mode >= 0 && mode <= 2, "mode 0, 1 or 2");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t o = 0;
    for (Layer& ly : m->L) {
        const size_t nw = (size_t)ly.n_out * ly.n_in;
        if (mode == 1) {
            SBR_TRY_CUDA(cudaMemcpyAsync(ly.W, params + o, nw * 4, cudaMemcpyDeviceToDevice, s));
            SBR_TRY_CUDA(cudaMemcpyAsync(ly.b, params + o + nw, ly.n_out * 4, cudaMemcpyDeviceToDevice, s));
        } else {
            const float* w = mode == 0 ? ly.W : ly.gW;
            const float* b = mode == 0 ? ly.b : ly.gb;
            SBR_TRY_CUDA(cudaMemcpyAsync(params + o, w, nw * 4, cudaMemcpyDeviceToDevice, s));
            SBR_TRY_CUDA(cudaMemcpyAsync(params + o + nw, b, ly.n_out * 4, cudaMemcpyDeviceToDevice, s));
        }
        o += (int64_t)nw + ly.n_out;
    }
    if (mode == 1) SBR_TRY(sync_bf16(m, s));
    return SBR_OK;
}

sbr_status sbr_mlp_status(const sbr_mlp* m) {
    clear_error();
    SBR_CHECK_ARG(m != nullptr, "mlp");
    unsigned bits = 0;
    SBR_TRY_CUDA(cudaDeviceSynchronize());
    SBR_TRY_CUDA(cudaMemcpy(&bits, m->status, 4, cudaMemcpyDeviceToHost));
    return status_from_bits(bits);
}

sbr_status sbr_mlp_set_lr(sbr_mlp* m, float lr) {
    clear_error();
    SBR_CHECK_ARG(m != nullptr && lr > 0.f && std::isfinite(lr), "mlp and lr > 0");
    m->cfg.lr = lr;
    return SBR_OK;
}

void sbr_mlp_free(sbr_mlp* m) { free_mlp(m); }

}  // extern "C"
