// FP32 batch instantiations, 16 warps per CTA.
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp32_batch() {
    cudaError_t e;
    if ((e = configure_batch<float, 2, 16>()) != cudaSuccess) return e;
    if ((e = configure_batch<float, 4, 16>()) != cudaSuccess) return e;
    if ((e = configure_batch<float, 8, 16>()) != cudaSuccess) return e;
    return configure_batch<float, 16, 16>();
}

cudaError_t launch_batch_fp32(const BatchArgs& a, int B, Schedule sc, int sm_count, cudaStream_t stream) {
    if (sc.warps != 16) return launch_batch_fp32_sched(a, B, sc, sm_count, stream);
    switch (B) {
        case 2: return launch_batch_t<float, 2, 16>(a, sm_count, stream);
        case 4: return launch_batch_t<float, 4, 16>(a, sm_count, stream);
        case 8: return launch_batch_t<float, 8, 16>(a, sm_count, stream);
        case 16: return launch_batch_t<float, 16, 16>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
