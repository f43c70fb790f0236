// FP32 iteration with the forward and the inverse transform on tensor cores
// (precision study): TF32 or BF16 hi/lo split products, FP32 accumulation;
// B = 4, 9 warps per CTA (shared memory: the DFT matrix table and a dense
// 8 KB coefficient array per warp besides the W rows).
#include "fsr_launch.h"

namespace fsrk {
namespace {

constexpr int kWarpsTc = 9;

template <Dft D>
size_t tc_smem() {
    return SmemLayout<float>::bytes(kWarpsTc) + TcTable<D>::bytes + sizeof(float2) * S * S * kWarpsTc;
}

template <Dft D>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_blocks_kernel<float, 4, kWarpsTc, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem<D>());
}

template <Dft D>
cudaError_t launch_one(const KernelArgs& a, int sm_count, cudaStream_t stream) {
    const size_t smem = tc_smem<D>();
    int grid = 0;
    cudaError_t e = persistent_grid(fsr_blocks_kernel<float, 4, kWarpsTc, D>, kWarpsTc, smem, a.nblocks, sm_count, &grid);
    if (e != cudaSuccess) return e;
    fsr_blocks_kernel<float, 4, kWarpsTc, D><<<grid, kWarpsTc * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_fp32_tc() {
    cudaError_t e = configure_one<Dft::TF32>();
    if (e != cudaSuccess) return e;
    return configure_one<Dft::BF16X3>();
}

cudaError_t launch_single_fp32_tc(const KernelArgs& a, int B, int bf16x3, int sm_count, cudaStream_t stream) {
    if (B != 4) return cudaErrorNotSupported;
    return bf16x3 ? launch_one<Dft::BF16X3>(a, sm_count, stream) : launch_one<Dft::TF32>(a, sm_count, stream);
}

}  // namespace fsrk
