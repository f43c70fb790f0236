// Wavefront kernel instantiations of the re-use form: FP32, B = 8 and 16.
#include "fsr_reuse.cuh"

namespace fsrk {

cudaError_t configure_reuse_f32hi() {
    cudaError_t e;
    if ((e = reuse::configure_b<float, 8>()) != cudaSuccess) return e;
    if ((e = reuse::configure_b<float, 16>()) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_reuse_f32hi(const ReuseLaunch& a, int B, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 8: return reuse::launch_b<float, 8>(a, sm_count, stream);
        case 16: return reuse::launch_b<float, 16>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
