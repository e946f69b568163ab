// Host-side launchers of the three instantiations of the persistent engine.
#pragma once

#include <cuda_runtime.h>

#include "engine.cuh"

namespace fde {

struct KernelInfo {
    int blocks_per_sm;
    int static_smem;
};

// Sets the dynamic shared-memory attribute and reports occupancy.
cudaError_t engine_prepare(int mode, int smem_bytes, KernelInfo* info);
cudaError_t engine_launch(int mode, const EngineArgs& a, int grid, cudaStream_t s);

cudaError_t engine_prepare_f64(int smem_bytes, KernelInfo* info);
cudaError_t engine_prepare_f32(int smem_bytes, KernelInfo* info);
cudaError_t engine_prepare_ir(int smem_bytes, KernelInfo* info);
cudaError_t engine_launch_f64(const EngineArgs& a, int grid, cudaStream_t s);
cudaError_t engine_launch_f32(const EngineArgs& a, int grid, cudaStream_t s);
cudaError_t engine_launch_ir(const EngineArgs& a, int grid, cudaStream_t s);

}  // namespace fde
