// Re-use of reconstructed pixels (the sequential form of the original FSR
// that Sec. II leaves out): the wavefront kernel, FP32 and FP64, every B of
// the 32 x 32 support.  One warp per block of the wavefront.
#include "fsr_launch.h"

namespace fsrk {

namespace {

// Warps per CTA of the FP32 wavefront kernel.  A wavefront of one image
// holds at most (blocks per image row) / (ceil(L / B) + 1) blocks (96 on a
// 1080p frame at B = 4), far fewer than the SMs can hold, so the per-block
// latency sets the time: small CTAs spread the blocks over more SMs (1080p,
// K = 100, delta = 0.5: 145 ms per frame with 8 warps per CTA, 130 ms with 1,
// 119 ms with 2, 115 ms with 4).  A launch holding the wavefronts of many
// images takes CTAs of 8 warps once its blocks exceed what CTAs of 4 hold in
// one wave (3 per SM by shared memory, against 2 CTAs of 8 = 16 warps).
constexpr int kWarpsReuse = 4;
constexpr int kWarpsReuseWide = 8;
constexpr int kCtasPerSmReuse = 3;

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
    cfg.gridDim = dim3((unsigned)((a.total + WARPS - 1) / WARPS));
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

template <int B>
cudaError_t configure_fp32() {
    cudaError_t e = configure_one<float, B, kWarpsReuse>();
    return e != cudaSuccess ? e : configure_one<float, B, kWarpsReuseWide>();
}

template <int B>
cudaError_t launch_fp32(const ReuseLaunch& a, int sm_count, cudaStream_t stream) {
    if (a.total > kCtasPerSmReuse * kWarpsReuse * sm_count) return launch_one<float, B, kWarpsReuseWide>(a, stream);
    return launch_one<float, B, kWarpsReuse>(a, stream);
}

}  // namespace

cudaError_t configure_reuse() {
    cudaError_t e;
    if ((e = configure_fp32<2>()) != cudaSuccess) return e;
    if ((e = configure_fp32<4>()) != cudaSuccess) return e;
    if ((e = configure_fp32<8>()) != cudaSuccess) return e;
    if ((e = configure_fp32<16>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 2, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 4, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<double, 8, 4>()) != cudaSuccess) return e;
    return configure_one<double, 16, 4>();
}

cudaError_t launch_reuse(const ReuseLaunch& a, int B, int fp64, int sm_count, cudaStream_t stream) {
    if (a.total <= 0) return cudaSuccess;
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
        case 2: return launch_fp32<2>(a, sm_count, stream);
        case 4: return launch_fp32<4>(a, sm_count, stream);
        case 8: return launch_fp32<8>(a, sm_count, stream);
        case 16: return launch_fp32<16>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
