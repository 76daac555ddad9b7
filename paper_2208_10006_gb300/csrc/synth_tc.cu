// H(f) synthesis on the tcgen05 tensor cores (BF16 hi/lo split).
#include "sbr_internal.cuh"
#include "synth_common.cuh"

namespace sbr {

sbr_status synth_tc_run(const sbr_path_list*, const float2*, const double*, int32_t, const double*,
                        int32_t, const double*, int32_t, int32_t, float2*, cudaStream_t) {
    set_error("tensor-core synthesis not built yet");
    return SBR_ERR_UNSUPPORTED;
}

}  // namespace sbr
