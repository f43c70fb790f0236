// Re-use of reconstructed pixels (the sequential form of the original FSR
// that Sec. II leaves out): the wavefront kernel, FP32 and FP64, every B of
// the 32 x 32 support.  One warp per block of the wavefront; the launch
// shapes are in fsr_reuse.cuh.
#include "fsr_reuse.cuh"

namespace fsrk {

cudaError_t configure_reuse() {
    cudaError_t e;
    if ((e = configure_reuse_f32lo()) != cudaSuccess) return e;
    if ((e = configure_reuse_f32hi()) != cudaSuccess) return e;
    return configure_reuse_f64();
}

cudaError_t launch_reuse(const ReuseLaunch& a, int B, int fp64, int sm_count, cudaStream_t stream) {
    if (a.total <= 0) return cudaSuccess;
    if (fp64) return launch_reuse_f64(a, B, sm_count, stream);
    if (B == 2 || B == 4) return launch_reuse_f32lo(a, B, sm_count, stream);
    return launch_reuse_f32hi(a, B, sm_count, stream);
}

}  // namespace fsrk
