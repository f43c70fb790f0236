// The 24 x 24 support (B in {4, 8}) of the small-support kernel in
// fsr_small.cuh: lane patches of 3 rows x 6 columns.
#include "fsr_small.cuh"

namespace fsrk {

cudaError_t configure_small24() {
    using namespace small;
    cudaError_t e;
    if ((e = configure_one<float, 24, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<float, 24, 8>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 24, 4>()) != cudaSuccess) return e;
    return configure_one<double, 24, 8>();
}

cudaError_t launch_small24(const BatchArgs& a, int B, int fp64, int chunk, int sm_count, cudaStream_t stream) {
    using namespace small;
    if (B == 4) return fp64 ? launch_one<double, 24, 4>(a, chunk, sm_count, stream)
                            : launch_one<float, 24, 4>(a, chunk, sm_count, stream);
    if (B == 8) return fp64 ? launch_one<double, 24, 8>(a, chunk, sm_count, stream)
                            : launch_one<float, 24, 8>(a, chunk, sm_count, stream);
    return cudaErrorNotSupported;
}

}  // namespace fsrk
