// Re-use of reconstructed pixels (the sequential form of the original FSR
// that Sec. II leaves out): the wavefront kernel, FP32 and FP64, every B of
// the 32 x 32 support.  One warp per block of the wavefront.
#include "fsr_launch.h"

namespace fsrk {

namespace {

template <typename T, int B, int WARPS>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_reuse_kernel<T, B, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmemLayout<T>::bytes(WARPS));
}

template <typename T, int B, int WARPS>
cudaError_t launch_one(const ReuseLaunch& a, cudaStream_t stream) {
    const int grid = (a.count + WARPS - 1) / WARPS;
    fsr_reuse_kernel<T, B, WARPS><<<grid, WARPS * 32, SmemLayout<T>::bytes(WARPS), stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_reuse() {
    cudaError_t e;
    if ((e = configure_one<float, 2, kWarpsFp32>()) != cudaSuccess) return e;
    if ((e = configure_one<float, 4, kWarpsFp32>()) != cudaSuccess) return e;
    if ((e = configure_one<float, 8, kWarpsFp32>()) != cudaSuccess) return e;
    if ((e = configure_one<float, 16, kWarpsFp32>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 2, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 4, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 8, 4>()) != cudaSuccess) return e;
    return configure_one<double, 16, 4>();
}

cudaError_t launch_reuse(const ReuseLaunch& a, int B, int fp64, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    if (fp64) {
        switch (B) {
            case 2: return launch_one<double, 2, 4>(a, stream);
            case 4: return launch_one<double, 4, 4>(a, stream);
            case 8: return launch_one<double, 8, 4>(a, stream);
            case 16: return launch_one<double, 16, 4>(a, stream);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (B) {
        case 2: return launch_one<float, 2, kWarpsFp32>(a, stream);
        case 4: return launch_one<float, 4, kWarpsFp32>(a, stream);
        case 8: return launch_one<float, 8, kWarpsFp32>(a, stream);
        case 16: return launch_one<float, 16, kWarpsFp32>(a, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
