// Short-lived-CTA form of the FP32 batch kernel (one chunk per warp, grid
// sized to the work): the serving loop's launches, so that launches on its
// higher-priority stream get SMs as soon as running CTAs finish.
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp32_short() {
    cudaError_t e;
    if ((e = configure_batch<float, 2, kWarpsFp32, false, true>()) != cudaSuccess) return e;
    if ((e = configure_batch<float, 4, kWarpsFp32, false, true>()) != cudaSuccess) return e;
    if ((e = configure_batch<float, 8, kWarpsFp32, false, true>()) != cudaSuccess) return e;
    return configure_batch<float, 16, kWarpsFp32, false, true>();
}

cudaError_t launch_batch_fp32_short(const BatchArgs& a, int B, cudaStream_t stream) {
    switch (B) {
        case 2: return launch_batch_t<float, 2, kWarpsFp32, false, true>(a, 0, stream);
        case 4: return launch_batch_t<float, 4, kWarpsFp32, false, true>(a, 0, stream);
        case 8: return launch_batch_t<float, 8, kWarpsFp32, false, true>(a, 0, stream);
        case 16: return launch_batch_t<float, 16, kWarpsFp32, false, true>(a, 0, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
