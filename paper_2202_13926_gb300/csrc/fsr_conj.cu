// Conjugate-pair ablation of the S = 32 batch kernel (the original FSR's
// real model: the selected component and its conjugate are updated
// together), B = 4, FP32 and FP64.
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_conj() {
    cudaError_t e;
    if ((e = configure_batch<float, 4, kWarpsFp32, true>()) != cudaSuccess) return e;
    return configure_batch<double, 4, 4, true>();
}

cudaError_t launch_batch_conj(const BatchArgs& a, int fp64, int sm_count, cudaStream_t stream) {
    return fp64 ? launch_batch_t<double, 4, 4, true>(a, sm_count, stream)
                : launch_batch_t<float, 4, kWarpsFp32, true>(a, sm_count, stream);
}

}  // namespace fsrk
