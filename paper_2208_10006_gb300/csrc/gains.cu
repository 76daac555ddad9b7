// Complex path gain g_n(f) (Eq. 1, 3, 6-10), one thread per (path, frequency);
// the per-path arithmetic is path_gain (gains.cuh). FP64 because the co-polar
// projection of a multi-bounce field can cancel to 1e-5 of the field, below
// which FP32 rounding alone exceeds a 1e-4 relative error on the gain; the
// work is P x F, negligible next to the trace.
#include <algorithm>

#include "gains.cuh"

namespace sbr {
namespace {

__global__ void k_gains(int64_t P, int32_t F, const int32_t* __restrict__ nb,
                        const int32_t* __restrict__ surf, const double* __restrict__ L,
                        const double* __restrict__ jones, const sbr_material* __restrict__ mats,
                        int32_t S, const double* __restrict__ freqs, const float* __restrict__ gamma,
                        const float* __restrict__ disp, int pol, float2* __restrict__ g) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * F) return;
    int64_t p = t / F;
    int32_t fi = (int32_t)(t - p * F);
    g[t] = path_gain(nb[p], surf + p * kKmax, L[p], jones + p * kJones, mats, S, freqs[fi],
                     gamma ? gamma + fi : nullptr, disp ? disp + fi : nullptr, pol);
}

}  // namespace

sbr_status gains_run(const sbr_path_list* pl, const sbr_material* mats, int32_t S,
                     const double* freqs, int32_t F, const float* gamma, const float* disp,
                     int32_t pol, float2* g, cudaStream_t s) {
    int64_t n = pl->P * (int64_t)F;
    if (n == 0) return SBR_OK;
    // small blocks: the per-(path, frequency) FP64 chains are latency-bound, spread them over every SM
    ::sbr::note_launch(), k_gains<<<(unsigned)((n + 63) / 64), 64, 0, s>>>(pl->P, F, pl->nb, pl->surf, pl->L, pl->jones,
                                                          mats, S, freqs, gamma, disp, pol, g);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

}  // namespace sbr
