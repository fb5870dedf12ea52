// Kernel launches, optionally with programmatic dependent launch (PDL).  Every kernel of the
// library starts with pdl_begin(): it lets the next kernel in the stream launch (its CTAs fill
// SMs as this grid drains) and then waits until the previous grid has completed and its writes
// are visible, so nothing is read early.  Without the launch attribute both instructions are
// no-ops, which is the default (pdl_enabled).
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace ufg {

// PDL for the launches of standalone operator calls (a PdlScope alive on the calling thread),
// and for every launch with UFG_PDL=1; the solvers' launches go without (measured slower on the
// batched solve).
bool pdl_enabled();
struct PdlScope {
  PdlScope();
  ~PdlScope();
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};

__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// kern<<<grid, block, smem, st>>>(args...) with the PDL attribute (and an optional cluster size).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, int cluster, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (cluster > 1) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)cluster;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  if (pdl_enabled()) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = na ? at : nullptr;
  cfg.numAttrs = (unsigned)na;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace ufg
