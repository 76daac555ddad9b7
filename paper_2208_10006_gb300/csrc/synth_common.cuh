// Shared prologue of the H(f) synthesis forms: per-element delays of the
// paths of one receiver and their delay-reduced weights (FP64).
#pragma once
#include "sbr_internal.cuh"

namespace sbr {

struct SynthPrep {
    int32_t Pr = 0;           // paths of the receiver
    int32_t off = 0;          // first path index in the path list
    const int32_t* nb0 = nullptr;  // device: reflections of the receiver's first path
                                   // (0 = it is the LoS path, which sorts first)
    double* dt = nullptr;     // [Pr * Nt]  |T_p - P1| - |T_0 - P1|
    double* dr = nullptr;     // [Pr * Nr]  |R_q - Pm| - |R_0 - Pm|
    double2* w = nullptr;     // [F * Pr]   g_n(f) exp(-j 2 pi frac(f L_n / c))
    double* dlos = nullptr;   // [Nr * Nt]  |T_p - R_q| - |T_0 - R_0|
};

sbr_status synth_prepare(const sbr_path_list* pl, const float2* g, const double* freqs, int32_t F,
                         const double* tx_elem, int32_t Nt, const double* rx_elem, int32_t Nr,
                         int32_t rx_index, SynthPrep* sp, cudaStream_t s);
void synth_release(SynthPrep* sp, cudaStream_t s);

}  // namespace sbr
