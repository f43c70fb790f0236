// Launchers of the per-block FSR kernels (one per arithmetic type).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "fsr_block.cuh"

namespace fsrk {

// Sets the dynamic shared-memory limit of every instantiation; call once per
// device with that device current.  Returns cudaSuccess or the first error.
cudaError_t configure_fp32();
cudaError_t configure_fp64();

// Enqueue the reconstruction of a.nblocks blocks with target size B on
// `stream`, on a persistent grid sized from the SM count.
cudaError_t launch_fp32(const KernelArgs& a, int B, int sm_count, cudaStream_t stream);
cudaError_t launch_fp64(const KernelArgs& a, int B, int sm_count, cudaStream_t stream);

}  // namespace fsrk
