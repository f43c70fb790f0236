// Re-use of reconstructed pixels (the sequential form of the original FSR
// that Sec. II leaves out): launch shapes of the wavefront kernel
// (fsr_reuse_kernel of fsr_block.cuh), instantiated in fsr_reuse_f32lo.cu
// (FP32, B = 2, 4), fsr_reuse_f32hi.cu (FP32, B = 8, 16) and fsr_reuse_f64.cu
// (FP64), so that the instantiations compile in parallel.
#pragma once

#include "fsr_launch.h"

namespace fsrk {
namespace reuse {

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

template <typename T, int B, int WARPS, int NSEG>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_reuse_kernel<T, B, WARPS, NSEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmemLayout<T>::bytes(WARPS));
}

// One wavefront, launched with programmatic stream serialization: its CTAs
// may start (and build their tables) while the previous wavefront runs; the
// kernel waits for that wavefront's completion before it reads any pixel.
// 1080p, K = 100, delta = 0.5, 4 warps per CTA: 115.8 ms per frame with
// plain stream order, 103.8 ms with this launch (outputs bit-identical).
template <typename T, int B, int WARPS, int NSEG>
cudaError_t launch_one(const ReuseLaunchN<NSEG>& a, cudaStream_t stream) {
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
    return cudaLaunchKernelEx(&cfg, fsr_reuse_kernel<T, B, WARPS, NSEG>, a);
}

// instantiated forms: one image in CTAs of 4 warps; up to kReuseSegs images
// in CTAs of 4, or of 8 for FP32 launches beyond one wave of CTAs of 4
template <typename T, int B>
cudaError_t configure_b() {
    cudaError_t e;
    if ((e = configure_one<T, B, kWarpsReuse, 1>()) != cudaSuccess) return e;
    if ((e = configure_one<T, B, kWarpsReuse, kReuseSegs>()) != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) return configure_one<T, B, kWarpsReuseWide, kReuseSegs>();
    return cudaSuccess;
}

template <typename T, int B>
cudaError_t launch_b(const ReuseLaunch& a, int sm_count, cudaStream_t stream) {
    if constexpr (sizeof(T) == 4) {
        if (a.total > kCtasPerSmReuse * kWarpsReuse * sm_count)
            return launch_one<T, B, kWarpsReuseWide, kReuseSegs>(a, stream);
    }
    if (a.nseg == 1) return launch_one<T, B, kWarpsReuse, 1>(one_image(a), stream);
    return launch_one<T, B, kWarpsReuse, kReuseSegs>(a, stream);
}

}  // namespace reuse

// per translation unit: configure / launch the instantiations of its B values
cudaError_t configure_reuse_f32lo();
cudaError_t launch_reuse_f32lo(const ReuseLaunch& a, int B, int sm_count, cudaStream_t stream);
cudaError_t configure_reuse_f32hi();
cudaError_t launch_reuse_f32hi(const ReuseLaunch& a, int B, int sm_count, cudaStream_t stream);
cudaError_t configure_reuse_f64();
cudaError_t launch_reuse_f64(const ReuseLaunch& a, int B, int sm_count, cudaStream_t stream);

}  // namespace fsrk
