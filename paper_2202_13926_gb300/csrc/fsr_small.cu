// Small supports S in {8, 16} (the kernel is in fsr_small.cuh); S = 24 is
// instantiated in fsr_small24.cu, S = 4 (a half-warp per block) is in
// fsr_tiny.cu, and FP32 at S = 16 runs the half-warp FFT kernel of
// fsr_s16.cu (FP64 at S = 16 runs the kernel of fsr_small.cuh).
#include "fsr_small.cuh"

namespace fsrk {

cudaError_t configure_small24();
cudaError_t launch_small24(const BatchArgs& a, int B, int fp64, int chunk, int sm_count, cudaStream_t stream);
cudaError_t launch_tiny(const BatchArgs& a, int B, int fp64, int chunk, int sm_count, cudaStream_t stream);
cudaError_t configure_s16();
cudaError_t launch_s16(const BatchArgs& a, int B, int chunk, int sm_count, cudaStream_t stream);

namespace {

// S = 16 is instantiated here for FP64 only (FP32 runs fsr_s16.cu).
template <typename T>
cudaError_t configure_all() {
    using namespace small;
    cudaError_t e;
    if constexpr (sizeof(T) == 8) {
        if ((e = configure_one<T, 16, 2>()) != cudaSuccess) return e;
        if ((e = configure_one<T, 16, 4>()) != cudaSuccess) return e;
        if ((e = configure_one<T, 16, 8>()) != cudaSuccess) return e;
    }
    if ((e = configure_one<T, 8, 2>()) != cudaSuccess) return e;
    return configure_one<T, 8, 4>();
}

template <typename T>
cudaError_t launch_any(const BatchArgs& a, int S, int B, int chunk, int sm_count, cudaStream_t stream) {
    using namespace small;
    if constexpr (sizeof(T) == 8) {
        if (S == 16 && B == 2) return launch_one<T, 16, 2>(a, chunk, sm_count, stream);
        if (S == 16 && B == 4) return launch_one<T, 16, 4>(a, chunk, sm_count, stream);
        if (S == 16 && B == 8) return launch_one<T, 16, 8>(a, chunk, sm_count, stream);
    }
    if (S == 8 && B == 2) return launch_one<T, 8, 2>(a, chunk, sm_count, stream);
    if (S == 8 && B == 4) return launch_one<T, 8, 4>(a, chunk, sm_count, stream);
    return cudaErrorNotSupported;
}

}  // namespace

bool small_supported(int S, int B) {
    return (S == 24 && (B == 4 || B == 8)) || (S == 16 && (B == 2 || B == 4 || B == 8)) ||
           (S == 8 && (B == 2 || B == 4)) || (S == 4 && (B == 2 || B == 4));
}

cudaError_t configure_small() {
    cudaError_t e = configure_all<float>();
    if (e != cudaSuccess) return e;
    if ((e = configure_all<double>()) != cudaSuccess) return e;
    if ((e = configure_s16()) != cudaSuccess) return e;
    return configure_small24();
}

cudaError_t launch_batch_small(const BatchArgs& a, int S, int B, int fp64, int chunk, int sm_count,
                               cudaStream_t stream) {
    if (S == 24) return launch_small24(a, B, fp64, chunk, sm_count, stream);
    if (S == 4) return launch_tiny(a, B, fp64, chunk, sm_count, stream);
    if (S == 16 && !fp64) return launch_s16(a, B, chunk, sm_count, stream);
    return fp64 ? launch_any<double>(a, S, B, chunk, sm_count, stream)
                : launch_any<float>(a, S, B, chunk, sm_count, stream);
}

}  // namespace fsrk
