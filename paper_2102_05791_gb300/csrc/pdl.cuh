// Programmatic dependent launch (PDL) for the kernels of the CG loop.
//
// A kernel launched with programmatic stream serialisation may start while
// its predecessor in the stream is still running.  griddepcontrol.wait then
// blocks until the predecessor grid has completed and its memory is
// visible; griddepcontrol.launch_dependents lets the successor be scheduled
// early.  Both are no-ops for kernels launched normally.  Every CG-loop
// kernel touches data written upstream only after pdl_wait(); the HVP tile
// kernel issues its bulk copies of static per-tile data before it, so those
// copies overlap the previous kernel.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace softsim {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch k<<<grid, block, smem, s>>>(args...), with programmatic stream
// serialisation when pdl is set.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

}  // namespace softsim
