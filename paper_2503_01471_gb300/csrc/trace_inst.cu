// The render kernel of two-level scenes (objects with their own BVHs under a
// per-environment BVH over the objects' boxes): 8x4 warp tiles, float32 nodes.
#include "trace_kernel.cuh"

namespace ags {

cudaError_t launch_trace_inst(const TraceArgs& a, int blocks, cudaStream_t s) {
  if (a.log2_tile_w != 3 || a.rays_per_lane != 1 || a.node_format != kNodeFp32 || a.slots || a.extra)
    return cudaErrorInvalidValue;
  k_trace_inst<<<blocks, kTraceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ags
