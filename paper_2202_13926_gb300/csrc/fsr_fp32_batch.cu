// FP32 batch instantiations (also the FP32 single-image path): kWarpsFp32 = 8
// warps per CTA, two CTAs per SM (8 x 13 KB of W rows + 8.4 KB of tables
// each, <= 128 registers per thread).
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp32_batch() {
    cudaError_t e;
    if ((e = configure_batch<float, 2, kWarpsFp32>()) != cudaSuccess) return e;
    if ((e = configure_batch<float, 4, kWarpsFp32>()) != cudaSuccess) return e;
    if ((e = configure_batch<float, 8, kWarpsFp32>()) != cudaSuccess) return e;
    return configure_batch<float, 16, kWarpsFp32>();
}

cudaError_t launch_batch_fp32(const BatchArgs& a, int B, Schedule sc, int sm_count, cudaStream_t stream) {
    if (sc.warps != kWarpsFp32) return launch_batch_fp32_sched(a, B, sc, sm_count, stream);
    switch (B) {
        case 2: return launch_batch_t<float, 2, kWarpsFp32>(a, sm_count, stream);
        case 4: return launch_batch_t<float, 4, kWarpsFp32>(a, sm_count, stream);
        case 8: return launch_batch_t<float, 8, kWarpsFp32>(a, sm_count, stream);
        case 16: return launch_batch_t<float, 16, kWarpsFp32>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

bool batch_schedule_supported(int fp64, int B, int warps) {
    if (B != 2 && B != 4 && B != 8 && B != 16) return false;
    if (fp64) return warps == 4;
    return warps == kWarpsFp32 || (B == 4 && (warps == 12 || warps == 16));
}

}  // namespace fsrk
