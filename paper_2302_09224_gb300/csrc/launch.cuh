// launch.cuh -- programmatic dependent launch for the solvers' kernel chains.
//
// Every kernel of a solver iteration depends on the one before it (alpha,
// beta and the vectors flow through device memory), so each used to start
// only after the previous grid had drained.  Launched with programmatic
// stream serialisation, a kernel's blocks are scheduled while its
// predecessor's last wave is still running; each kernel calls pdl_wait()
// before its first access to memory another kernel of the chain writes (the
// wait returns once the predecessor grid has completed and its writes are
// visible), then pdl_launch_dependents() so that its own successor can be
// scheduled in turn.  Launched without the attribute, both are no-ops.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <utility>

namespace hisq {

// 1: solver kernels are launched with programmatic stream serialisation
// (hisq_programmatic_launch switches it; read at every launch)
extern std::atomic<int> pdl_mode;

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// kernel<<<grid, block, 0, s>>>(args...) with programmatic stream
// serialisation when pdl_mode is on
template <typename... P, typename... A>
inline cudaError_t launch_chained(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t s, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = pdl_mode.load(std::memory_order_relaxed) ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace hisq
