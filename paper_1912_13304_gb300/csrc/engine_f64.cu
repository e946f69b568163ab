// Instantiation of the persistent engine for mode kModeF64.
#include "launch.h"

namespace fde {

cudaError_t engine_prepare_f64(int smem_bytes, KernelInfo* info) {
    cudaError_t e = cudaFuncSetAttribute(fde_engine<kModeF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fde_engine<kModeF64>);
    if (e != cudaSuccess) return e;
    info->static_smem = (int)fa.sharedSizeBytes;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&info->blocks_per_sm, fde_engine<kModeF64>, kThreads,
                                                         smem_bytes);
}

cudaError_t engine_launch_f64(const EngineArgs& a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = a.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fde_engine<kModeF64>, a);
}

}  // namespace fde
