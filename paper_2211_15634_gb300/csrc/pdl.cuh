// Programmatic dependent launch (sm_90 and later).
//
// A kernel launched with launch_pdl may begin while the kernel before it on the
// same stream is still running: its CTAs are scheduled once every CTA of that
// kernel has executed grid_dep_launch() (or exited), so their set-up (shared
// memory, mbarriers) overlaps the previous kernel's last wave and the launch gap
// disappears.  grid_dep_wait() blocks the calling thread until the previous kernel
// has completed and its memory operations are visible, so every thread of a kernel
// launched this way calls it before its first global memory access - read or
// write, TMA included (the previous step may still read the buffer this one writes).
// In a kernel launched without the attribute both are no-ops.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace psd {

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// kern<<<grid, block, smem, s>>>(args...) with programmatic stream serialization.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace psd
