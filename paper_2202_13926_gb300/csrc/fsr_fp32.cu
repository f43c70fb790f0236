// FP32 single-image instantiations (the production path): 12 warps per CTA,
// one CTA per SM (12 x 17.2 KB of W rows + 8.4 KB of tables).
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp32() {
    cudaError_t e;
    if ((e = configure_single<float, 2, 12>()) != cudaSuccess) return e;
    if ((e = configure_single<float, 4, 12>()) != cudaSuccess) return e;
    if ((e = configure_single<float, 8, 12>()) != cudaSuccess) return e;
    return configure_single<float, 16, 12>();
}

cudaError_t launch_single_fp32(const KernelArgs& a, int B, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 2: return launch_single_t<float, 2, 12>(a, sm_count, stream);
        case 4: return launch_single_t<float, 4, 12>(a, sm_count, stream);
        case 8: return launch_single_t<float, 8, 12>(a, sm_count, stream);
        case 16: return launch_single_t<float, 16, 12>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

bool batch_schedule_supported(int fp64, int B, int warps) {
    if (B != 2 && B != 4 && B != 8 && B != 16) return false;
    if (fp64) return warps == 4;
    return warps == 12 || (B == 4 && (warps == 4 || warps == 6));
}

}  // namespace fsrk
