// FP64 instantiations (debug arithmetic whose selection sequences are compared
// with an FP64 reference): 4 warps per CTA (4 x 34 KB of W rows + 17 KB tables).
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp64() {
    cudaError_t e;
    if ((e = configure_single<double, 2, 4>()) != cudaSuccess) return e;
    if ((e = configure_single<double, 4, 4>()) != cudaSuccess) return e;
    if ((e = configure_single<double, 8, 4>()) != cudaSuccess) return e;
    return configure_single<double, 16, 4>();
}

cudaError_t launch_single_fp64(const KernelArgs& a, int B, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 2: return launch_single_t<double, 2, 4>(a, sm_count, stream);
        case 4: return launch_single_t<double, 4, 4>(a, sm_count, stream);
        case 8: return launch_single_t<double, 8, 4>(a, sm_count, stream);
        case 16: return launch_single_t<double, 16, 4>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
