// pdl.cuh -- programmatic dependent launch for chains of dependent kernels.
//
// A kernel launched with launch_pdl may be scheduled before the kernel ahead
// of it on the stream has finished (once every CTA of that kernel has called
// pdl_release, or has exited), so that its launch is not paid between the
// two. Every such kernel calls pdl_wait before it touches memory that an
// earlier kernel writes: the wait returns when all earlier work on the stream
// has completed and its writes are visible, which is the order a plain
// launch gives. pdl_release lets the next kernel be scheduled; it says
// nothing about this kernel's own writes, which the next kernel's pdl_wait
// covers. Both are no-ops for a kernel launched the plain way.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace synth {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Records that a kernel which releases its successor at its start was
// launched on st: a fused render that follows it then waits for it as for
// any kernel (the fused render overlaps only another fused render whose
// buffers it does not share; render_fused.cu keeps that record).
void note_early_release_launch(cudaStream_t st);

// kernel<<<grid, block, smem, st>>>(args...) with the programmatic
// stream-serialization attribute.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
  note_early_release_launch(st);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace synth
