// FP32 iteration with the forward and the inverse transform on the tensor
// cores (precision study): TF32 or BF16 hi/lo split products on tcgen05.mma
// with FP32 accumulators in tensor memory; B = 4, one CTA of kWarpsTc warps
// per SM (W rows, the DFT matrix table and the pick lists in shared memory,
// all 512 tensor-memory columns).
#include "fsr_launch.h"
#include "fsr_tc5.cuh"

namespace fsrk {
namespace {

template <Dft D>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_tc_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcLayout::bytes);
}

template <Dft D>
cudaError_t launch_one(const KernelArgs& a, int sm_count, cudaStream_t stream) {
    int grid = 0;
    cudaError_t e = persistent_grid(fsr_tc_kernel<D>, kWarpsTc, TcLayout::bytes, a.nblocks, sm_count, &grid);
    if (e != cudaSuccess) return e;
    fsr_tc_kernel<D><<<grid, kWarpsTc * 32, TcLayout::bytes, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_fp32_tc() {
    cudaError_t e = configure_one<Dft::TF32>();
    if (e != cudaSuccess) return e;
    return configure_one<Dft::BF16X3>();
}

cudaError_t launch_single_fp32_tc(const KernelArgs& a, int B, int bf16x3, int sm_count, cudaStream_t stream) {
    if (B != 4 || a.im.K > kTcMaxIters) return cudaErrorNotSupported;
    return bf16x3 ? launch_one<Dft::BF16X3>(a, sm_count, stream) : launch_one<Dft::TF32>(a, sm_count, stream);
}

}  // namespace fsrk
