// Re-use of reconstructed pixels (the sequential form of the original FSR
// that Sec. II leaves out): the wavefront kernel, FP32 and FP64, every B of
// the 32 x 32 support.  One warp per block of the wavefront.
#include "fsr_launch.h"

namespace fsrk {

namespace {

// Warps per CTA of the FP32 wavefront kernel.  A wavefront holds at most
// (blocks per image row) / (ceil(L / B) + 1) blocks (96 on a 1080p frame at
// B = 4), far fewer than the SMs can hold, so the per-block latency sets the time: small
// CTAs spread the blocks over more SMs.  1080p, K = 100, delta = 0.5: 145 ms
// per frame with 8 warps per CTA, 130 ms with 1, 119 ms with 2, 115 ms with 4.
constexpr int kWarpsReuse = 4;

template <typename T, int B, int WARPS>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_reuse_kernel<T, B, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmemLayout<T>::bytes(WARPS));
}

// One wavefront, launched with programmatic stream serialization: its CTAs
// may start (and build their tables) while the previous wavefront runs; the
// kernel waits for that wavefront's completion before it reads any pixel.
// 1080p, K = 100, delta = 0.5, 4 warps per CTA: 115.8 ms per frame with
// plain stream order, 103.8 ms with this launch (outputs bit-identical).
template <typename T, int B, int WARPS>
cudaError_t launch_one(const ReuseLaunch& a, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((a.count + WARPS - 1) / WARPS));
    cfg.blockDim = dim3(WARPS * 32);
    cfg.dynamicSmemBytes = SmemLayout<T>::bytes(WARPS);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fsr_reuse_kernel<T, B, WARPS>, a);
}

}  // namespace

cudaError_t configure_reuse() {
    cudaError_t e;
    if ((e = configure_one<float, 2, kWarpsReuse>()) != cudaSuccess) return e;
    if ((e = configure_one<float, 4, kWarpsReuse>()) != cudaSuccess) return e;
    if ((e = configure_one<float, 8, kWarpsReuse>()) != cudaSuccess) return e;
    if ((e = configure_one<float, 16, kWarpsReuse>()) != cudaSuccess) return e;
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
        case 2: return launch_one<float, 2, kWarpsReuse>(a, stream);
        case 4: return launch_one<float, 4, kWarpsReuse>(a, stream);
        case 8: return launch_one<float, 8, kWarpsReuse>(a, stream);
        case 16: return launch_one<float, 16, kWarpsReuse>(a, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
