// Wavefront kernel instantiations of the re-use form: FP64 debug arithmetic, every B.
#include "fsr_reuse.cuh"

namespace fsrk {

cudaError_t configure_reuse_f64() {
    cudaError_t e;
    if ((e = reuse::configure_b<double, 2>()) != cudaSuccess) return e;
    if ((e = reuse::configure_b<double, 4>()) != cudaSuccess) return e;
    if ((e = reuse::configure_b<double, 8>()) != cudaSuccess) return e;
    if ((e = reuse::configure_b<double, 16>()) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_reuse_f64(const ReuseLaunch& a, int B, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 2: return reuse::launch_b<double, 2>(a, sm_count, stream);
        case 4: return reuse::launch_b<double, 4>(a, sm_count, stream);
        case 8: return reuse::launch_b<double, 8>(a, sm_count, stream);
        case 16: return reuse::launch_b<double, 16>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
