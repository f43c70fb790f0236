// Launchers of the FSR kernels.  Each translation unit instantiates one
// arithmetic type / schedule family; fsr_capi.cu dispatches.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "fsr_block.cuh"

namespace fsrk {

// Warps per CTA of the default FP32 batch kernels (which also run every FP32
// single-image call): two CTAs of 8 warps per SM.
constexpr int kWarpsFp32 = 8;

// A persistent schedule: warps per CTA (one support block per warp) and the
// number of blocks a warp takes per work-counter increment (batch form).
struct Schedule {
    int warps;
    int chunk;
};

// Sets the dynamic shared-memory limit of every instantiation of the family;
// call once per device with that device current.
cudaError_t configure_fp32_batch();
cudaError_t configure_fp32_sched();
cudaError_t configure_fp64();
cudaError_t configure_fp64_batch();
cudaError_t configure_fp32_tc();

// Single image (FP64 debug, 4 warps per CTA): warps take blocks from a work counter.
cudaError_t launch_single_fp64(const KernelArgs& a, int B, int sm_count, cudaStream_t stream);
// Both 2-D DFTs on tensor cores (TF32, or BF16 hi/lo with bf16x3 = 1); B = 4 only.
cudaError_t launch_single_fp32_tc(const KernelArgs& a, int B, int bf16x3, int sm_count, cudaStream_t stream);

// Batch form.  Returns cudaErrorNotSupported for a schedule that is not
// instantiated (see batch_schedule_supported).
cudaError_t launch_batch_fp32(const BatchArgs& a, int B, Schedule sc, int sm_count, cudaStream_t stream);
cudaError_t launch_batch_fp32_sched(const BatchArgs& a, int B, Schedule sc, int sm_count, cudaStream_t stream);
cudaError_t launch_batch_fp64(const BatchArgs& a, int B, Schedule sc, int sm_count, cudaStream_t stream);

// Small supports S in {4, 8, 16, 24} (FP32 and FP64, batch-table interface):
// S = 24 with B in {4, 8}, S = 16 with B in {2, 4, 8}, S = 8 and S = 4 with
// B in {2, 4}.
bool small_supported(int S, int B);
cudaError_t configure_small();
cudaError_t launch_batch_small(const BatchArgs& a, int S, int B, int fp64, int chunk, int sm_count,
                               cudaStream_t stream);

// Short-lived-CTA form of the FP32 batch kernel (kWarpsFp32 warps, any B),
// for launches with a.one_round set (the serving loop).
cudaError_t configure_fp32_short();
cudaError_t launch_batch_fp32_short(const BatchArgs& a, int B, cudaStream_t stream);

// Conjugate-pair ablation (S = 32, B = 4; FP32 with kWarpsFp32 warps per
// CTA, FP64 with 4), batch-table interface.
cudaError_t configure_conj();
cudaError_t launch_batch_conj(const BatchArgs& a, int fp64, int sm_count, cudaStream_t stream);

// Re-use of reconstructed pixels: one wavefront launch (FP32 with
// kWarpsFp32 warps per CTA, FP64 with 4), any B of S = 32.
cudaError_t configure_reuse();
cudaError_t launch_reuse(const ReuseLaunch& a, int B, int fp64, int sm_count, cudaStream_t stream);

// Warps-per-CTA values instantiated for (precision, B): FP32 has 8 for every
// B and also 12 and 16 for B = 4; FP64 has 4.
bool batch_schedule_supported(int fp64, int B, int warps);

// Persistent grid: resident CTAs per SM x SMs, capped by the work available.
template <typename Kernel>
cudaError_t persistent_grid(Kernel k, int warps, size_t smem, long long work_warps, int sm_count, int* grid) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long need = (work_warps + warps - 1) / warps;
    long long g = (long long)sm_count * per_sm;
    if (need < g) g = need;
    if (g < 1) g = 1;
    *grid = (int)g;
    return cudaSuccess;
}

template <typename T, int B, int WARPS>
cudaError_t configure_single() {
    return cudaFuncSetAttribute(fsr_blocks_kernel<T, B, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmemLayout<T>::bytes(WARPS));
}

template <typename T, int B, int WARPS, bool CONJ = false, bool ONE_ROUND = false>
cudaError_t configure_batch() {
    return cudaFuncSetAttribute(fsr_batch_kernel<T, B, WARPS, CONJ, ONE_ROUND>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SmemLayout<T>::bytes(WARPS));
}

template <typename T, int B, int WARPS>
cudaError_t launch_single_t(const KernelArgs& a, int sm_count, cudaStream_t stream) {
    const size_t smem = SmemLayout<T>::bytes(WARPS);
    int grid = 0;
    cudaError_t e = persistent_grid(fsr_blocks_kernel<T, B, WARPS>, WARPS, smem, a.nblocks, sm_count, &grid);
    if (e != cudaSuccess) return e;
    fsr_blocks_kernel<T, B, WARPS><<<grid, WARPS * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

template <typename T, int B, int WARPS, bool CONJ = false, bool ONE_ROUND = false>
cudaError_t launch_batch_t(const BatchArgs& a, int sm_count, cudaStream_t stream) {
    const size_t smem = SmemLayout<T>::bytes(WARPS);
    int grid = 0;
    cudaError_t e = cudaSuccess;
    if constexpr (ONE_ROUND) {   // short-lived CTAs: one chunk per warp
        const long long per_cta = (long long)WARPS * a.chunk;
        const long long g = (a.total + per_cta - 1) / per_cta;
        grid = (int)(g < 1 ? 1 : (g > 0x7fffffffll ? 0x7fffffffll : g));
    } else {
        e = persistent_grid(fsr_batch_kernel<T, B, WARPS, CONJ>, WARPS, smem, a.total, sm_count, &grid);
    }
    if (e != cudaSuccess) return e;
    fsr_batch_kernel<T, B, WARPS, CONJ, ONE_ROUND><<<grid, WARPS * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace fsrk
