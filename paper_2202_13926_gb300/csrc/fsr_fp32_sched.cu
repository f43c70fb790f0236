// FP32 batch kernels with other CTA shapes for the schedule autotuner, B = 4:
// 12 warps (one CTA per SM, up to 168 registers) and 16 warps (one CTA per
// SM, 128 registers).
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp32_sched() {
    cudaError_t e;
    if ((e = configure_batch<float, 4, 12>()) != cudaSuccess) return e;
    return configure_batch<float, 4, 16>();
}

cudaError_t launch_batch_fp32_sched(const BatchArgs& a, int B, Schedule sc, int sm_count, cudaStream_t stream) {
    if (B != 4) return cudaErrorNotSupported;
    switch (sc.warps) {
        case 12: return launch_batch_t<float, 4, 12>(a, sm_count, stream);
        case 16: return launch_batch_t<float, 4, 16>(a, sm_count, stream);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace fsrk
