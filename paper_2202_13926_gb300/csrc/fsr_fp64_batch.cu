// FP64 batch instantiations, 4 warps per CTA.
#include "fsr_launch.h"

namespace fsrk {

cudaError_t configure_fp64_batch() {
    cudaError_t e;
    if ((e = configure_batch<double, 2, 4>()) != cudaSuccess) return e;
    if ((e = configure_batch<double, 4, 4>()) != cudaSuccess) return e;
    if ((e = configure_batch<double, 8, 4>()) != cudaSuccess) return e;
    return configure_batch<double, 16, 4>();
}

cudaError_t launch_batch_fp64(const BatchArgs& a, int B, Schedule sc, int sm_count, cudaStream_t stream) {
    if (sc.warps != 4) return cudaErrorNotSupported;
    switch (B) {
        case 2: return launch_batch_t<double, 2, 4>(a, sm_count, stream);
        case 4: return launch_batch_t<double, 4, 4>(a, sm_count, stream);
        case 8: return launch_batch_t<double, 8, 4>(a, sm_count, stream);
        case 16: return launch_batch_t<double, 16, 4>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
