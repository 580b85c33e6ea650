// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may begin while the kernel before it in
// the stream is still running, so its launch latency overlaps that kernel's
// tail.  Such a kernel calls griddep_wait() before its first access to memory
// that the previous kernel writes (a hardware wait for that grid to complete
// and its writes to be visible, not a spin), and griddep_launch_dependents()
// once it has done its work, which lets the next such kernel be scheduled.
// Chains of short dependent kernels (the adjoint's passes, the multigrid
// levels) lose most of their launch gaps this way.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace hh {

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
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

}  // namespace hh
