// The render kernel with a short stack (16 or 32 entries, 8x4 tiles) and
// the retry pass that walks the rays whose stack ran out again with the full
// 64-entry stack (trace_kernel.cuh). Outputs equal those of k_trace.
#include "trace_kernel.cuh"

namespace ags {

namespace {
template <int kFmt>
cudaError_t launch_short_fmt(const TraceArgs& a, int blocks, int retry_blocks, cudaStream_t s) {
  if (a.stack_depth == 16) k_trace_short<kFmt, 16><<<blocks, kTraceThreads, 0, s>>>(a);
  else if (a.stack_depth == 32) k_trace_short<kFmt, 32><<<blocks, kTraceThreads, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_trace_retry<kFmt><<<retry_blocks, kTraceThreads, 0, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_trace_short(const TraceArgs& a, int blocks, int retry_blocks, cudaStream_t s) {
  if (a.log2_tile_w != 3 || a.rays_per_lane != 1 || a.slots || a.extra || a.instanced || !a.retry_list ||
      !a.retry_count)
    return cudaErrorInvalidValue;
  switch (a.node_format) {
    case kNodeFp32: return launch_short_fmt<kNodeFp32>(a, blocks, retry_blocks, s);
    case kNodeFp16: return launch_short_fmt<kNodeFp16>(a, blocks, retry_blocks, s);
    case kNodeQ8: return launch_short_fmt<kNodeQ8>(a, blocks, retry_blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ags
