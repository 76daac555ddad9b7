// Complex path gain g_n(f) (Eq. 1, 3, 6-10), one thread per (path, frequency);
// the per-path arithmetic is path_gain (gains.cuh). FP64 because the co-polar
// projection of a multi-bounce field can cancel to 1e-5 of the field, below
// which FP32 rounding alone exceeds a 1e-4 relative error on the gain; the
// work is P x F, negligible next to the trace.
#include <algorithm>

#include "gains.cuh"

namespace sbr {
namespace {

// Eight lanes per (path, frequency): lane k computes the coefficients of
// reflection k (the FP64 chains of the reflections run side by side), lane 0
// then carries the field through them in order and finishes the gain, with the
// arithmetic of path_gain (bit-identical results).
constexpr int kGainLanes = 8;
static_assert(kGainLanes >= kKmax, "one lane per reflection");
constexpr int kGainThreads = 64;

__global__ void __launch_bounds__(kGainThreads)
k_gains(int64_t P, int32_t F, const int32_t* __restrict__ nb, const int32_t* __restrict__ surf,
        const double* __restrict__ L, const double* __restrict__ jones, const sbr_material* __restrict__ mats,
        int32_t S, const double* __restrict__ freqs, const float* __restrict__ gamma,
        const float* __restrict__ disp, int pol, float2* __restrict__ g) {
    ::sbr::pdl_wait();
    __shared__ Refl s_rf[kGainThreads];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t item = t / kGainLanes;
    const int k = (int)(t % kGainLanes);
    const bool valid = item < P * F;
    const int64_t p = valid ? item / F : 0;
    const int32_t fi = valid ? (int32_t)(item - p * F) : 0;
    const int m = valid ? nb[p] : 0;
    const double f = valid ? freqs[fi] : 1.0;
    const double* J = jones + p * kJones;
    const int32_t* sp = surf + p * kKmax;
    if (k < m) {
        const int s = sp[k];
        if (s >= 0 && s < S) s_rf[threadIdx.x] = reflection(mats[s], J[36 + k], f);
    }
    __syncwarp();
    if (!valid || k != 0) return;
    // a surface id outside [0, S) (not reachable: S is checked on the host)
    for (int q = 0; q < m; ++q)
        if (sp[q] < 0 || sp[q] >= S) { g[item] = make_float2(NAN, NAN); return; }
    const int pb = pol == SBR_POL_V ? 0 : 2;
    cd b0{J[pb], 0.0}, b1{J[pb + 1], 0.0};
    for (int q = 0; q < m; ++q) reflect_field(b0, b1, s_rf[threadIdx.x + q], J, q, m);
    g[item] = finish_gain(b0, b1, J, pb, L[p], f, gamma ? gamma + fi : nullptr, disp ? disp + fi : nullptr);
}

}  // namespace

sbr_status gains_run(const sbr_path_list* pl, const sbr_material* mats, int32_t S,
                     const double* freqs, int32_t F, const float* gamma, const float* disp,
                     int32_t pol, float2* g, cudaStream_t s) {
    int64_t n = pl->P * (int64_t)F;
    if (n == 0) return SBR_OK;
    // small blocks of eight lanes per (path, frequency): the FP64 chains are
    // latency-bound, so they are spread over every SM and split by reflection
    const int64_t threads = n * kGainLanes;
    ::sbr::note_launch(), (void)::sbr::launch_pdl(k_gains, dim3((unsigned)((threads + kGainThreads - 1) / kGainThreads)), dim3(kGainThreads), 0, s,
        pl->P, F, pl->nb, pl->surf, pl->L, pl->jones, mats, S, freqs, gamma, disp, pol, g);
    SBR_TRY_CUDA(cudaGetLastError());
    return SBR_OK;
}

}  // namespace sbr
