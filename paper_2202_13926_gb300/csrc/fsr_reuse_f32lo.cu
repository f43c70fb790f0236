// Wavefront kernel instantiations of the re-use form: FP32, B = 2 and 4.
#include "fsr_reuse.cuh"

namespace fsrk {

cudaError_t configure_reuse_f32lo() {
    cudaError_t e;
    if ((e = reuse::configure_b<float, 2>()) != cudaSuccess) return e;
    if ((e = reuse::configure_b<float, 4>()) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_reuse_f32lo(const ReuseLaunch& a, int B, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 2: return reuse::launch_b<float, 2>(a, sm_count, stream);
        case 4: return reuse::launch_b<float, 4>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
