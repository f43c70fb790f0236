// Dispatch of the supports smaller than 32.  FP32 at S = 4, 8, 16 runs the
// group kernel of fsr_group.cu (a group of S lanes per block); S = 24 (FP32
// and FP64) runs the lane-patch kernel of fsr_small.cuh, instantiated in
// fsr_small24.cu; FP64 at S = 8 and 16 runs the same lane-patch kernel
// (instantiated here) and FP64 at S = 4 the half-warp kernel of fsr_tiny.cu.
#include "fsr_small.cuh"

namespace fsrk {

cudaError_t configure_small24();
cudaError_t launch_small24(const BatchArgs& a, int B, int fp64, int chunk, int sm_count, cudaStream_t stream);
cudaError_t launch_tiny(const BatchArgs& a, int B, int chunk, int sm_count, cudaStream_t stream);
cudaError_t configure_group();
cudaError_t launch_group(const BatchArgs& a, int S, int B, int chunk, int sm_count, cudaStream_t stream);

namespace {

// FP64 at S = 8 and 16
cudaError_t configure_patch_small() {
    using namespace small;
    cudaError_t e;
    if ((e = configure_one<double, 16, 2>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 16, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 16, 8>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 8, 2>()) != cudaSuccess) return e;
    return configure_one<double, 8, 4>();
}

cudaError_t launch_patch_small(const BatchArgs& a, int S, int B, int chunk, int sm_count, cudaStream_t stream) {
    using namespace small;
    if (S == 16 && B == 2) return launch_one<double, 16, 2>(a, chunk, sm_count, stream);
    if (S == 16 && B == 4) return launch_one<double, 16, 4>(a, chunk, sm_count, stream);
    if (S == 16 && B == 8) return launch_one<double, 16, 8>(a, chunk, sm_count, stream);
    if (S == 8 && B == 2) return launch_one<double, 8, 2>(a, chunk, sm_count, stream);
    if (S == 8 && B == 4) return launch_one<double, 8, 4>(a, chunk, sm_count, stream);
    return cudaErrorNotSupported;
}

}  // namespace

bool small_supported(int S, int B) {
    return (S == 24 && (B == 4 || B == 8)) || (S == 16 && (B == 2 || B == 4 || B == 8)) ||
           (S == 8 && (B == 2 || B == 4)) || (S == 4 && (B == 2 || B == 4));
}

cudaError_t configure_small() {
    cudaError_t e = configure_patch_small();
    if (e != cudaSuccess) return e;
    if ((e = configure_group()) != cudaSuccess) return e;
    return configure_small24();
}

cudaError_t launch_batch_small(const BatchArgs& a, int S, int B, int fp64, int chunk, int sm_count,
                               cudaStream_t stream) {
    if (S == 24) return launch_small24(a, B, fp64, chunk, sm_count, stream);
    if (!fp64 && (S == 4 || S == 8 || S == 16)) return launch_group(a, S, B, chunk, sm_count, stream);
    if (fp64 && S == 4) return launch_tiny(a, B, chunk, sm_count, stream);
    if (!fp64) return cudaErrorNotSupported;
    return launch_patch_small(a, S, B, chunk, sm_count, stream);
}

}  // namespace fsrk
