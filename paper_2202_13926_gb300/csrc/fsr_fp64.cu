// FP64 instantiations of the per-block FSR kernel (debug arithmetic: selection
// sequences comparable with an FP64 reference).
#include "fsr_launch.h"

namespace fsrk {
namespace {

constexpr int kWarps64 = 4;    // 4 x 33.8 KB of W rows + 16.9 KB tables per CTA

template <int B>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_blocks_kernel<double, B, kWarps64>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmemLayout<double>::bytes(kWarps64));
}

template <int B>
cudaError_t launch_one(const KernelArgs& a, int sm_count, cudaStream_t stream) {
    const size_t smem = SmemLayout<double>::bytes(kWarps64);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, fsr_blocks_kernel<double, B, kWarps64>, kWarps64 * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long need = (a.nblocks + kWarps64 - 1) / kWarps64;
    long long grid = (long long)sm_count * per_sm;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    fsr_blocks_kernel<double, B, kWarps64><<<(unsigned)grid, kWarps64 * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_fp64() {
    cudaError_t e;
    if ((e = configure_one<2>()) != cudaSuccess) return e;
    if ((e = configure_one<4>()) != cudaSuccess) return e;
    if ((e = configure_one<8>()) != cudaSuccess) return e;
    return configure_one<16>();
}

cudaError_t launch_fp64(const KernelArgs& a, int B, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 2: return launch_one<2>(a, sm_count, stream);
        case 4: return launch_one<4>(a, sm_count, stream);
        case 8: return launch_one<8>(a, sm_count, stream);
        case 16: return launch_one<16>(a, sm_count, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsrk
