// FP32 single-image instantiations (the production path): 16 warps per CTA,
// one CTA per SM (16 x 13 KB of W rows + 8.4 KB of tables, <= 128 registers).
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp32() {
    cudaError_t e;
    if ((e = configure_single<float, 2, 16>()) != cudaSuccess) return e;
    if ((e = configure_single<float, 4, 16>()) != cudaSuccess) return e;
    if ((e = configure_single<float, 8, 16>()) != cudaSuccess) return e;
    return configure_single<float, 16, 16>();
}

cudaError_t launch_single_fp32(const KernelArgs& a, int B, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 2: return launch_single_t<float, 2, 16>(a, sm_count, stream);
        case 4: return launch_single_t<float, 4, 16>(a, sm_count, stream);
        case 8: return launch_single_t<float, 8, 16>(a, sm_count, stream);
        case 16: return launch_single_t<float, 16, 16>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

bool batch_schedule_supported(int fp64, int B, int warps) {
    if (B != 2 && B != 4 && B != 8 && B != 16) return false;
    if (fp64) return warps == 4;
    return warps == 16 || (B == 4 && (warps == 8 || warps == 12));
}

}  // namespace fsrk
