// Batched ray casting (Sec. III-D.1: one ray per pixel tested against the
// environment's meshes M_{i,t}; range vs depth): the
// launch shapes of the plain render, the instrumented count and the serving
// slot mode. The kernel itself is in trace_kernel.cuh; the variants with
// extra work (hit channels, stereo shadows, ray tables) are instantiated in
// trace_extra.cu.
#include "trace_kernel.cuh"

namespace ags {
int trace_blocks_per_sm(bool count) {
  int n = 0;
  cudaError_t e =
      count ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<true, 8, 1, false, kNodeFp32>, kTraceThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<false, 8, 1, false, kNodeFp32>, kTraceThreads, 0);
  return (e == cudaSuccess && n > 0) ? n : 1;
}

bool trace_shape_supported(int tile_w, int rays_per_lane) {
  for (int k = 0; k < kTraceShapes; ++k)
    if (kTraceShape[k][0] == tile_w && kTraceShape[k][1] == rays_per_lane) return true;
  return false;
}

namespace {
template <int kFmt>
cudaError_t launch_fmt(const TraceArgs& a, int blocks, bool count, cudaStream_t s) {
  const int w = 1 << a.log2_tile_w, r = a.rays_per_lane;
  if (a.slots) {
    if (w == 8 && r == 1) k_trace<false, 8, 1, true, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
    else return cudaErrorInvalidValue;
  } else if (a.extra) {
    if (w != 8 || r != 1 || count) return cudaErrorInvalidValue;
    return launch_trace_extra(a, blocks, s);
  } else if (count) {
    k_trace<true, 8, 1, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else if (w == 8 && r == 1) {
    k_trace<false, 8, 1, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else if (w == 4 && r == 1) {
    k_trace<false, 4, 1, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else if (w == 8 && r == 2) {
    k_trace<false, 8, 2, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else if (w == 16 && r == 2) {
    k_trace<false, 16, 2, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else if (w == 16 && r == 4) {
    k_trace<false, 16, 4, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else if (w == 16 && r == 1) {
    k_trace<false, 16, 1, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else if (w == 32 && r == 1) {
    k_trace<false, 32, 1, false, kFmt><<<blocks, kTraceThreads, 0, s>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_trace(const TraceArgs& a, int blocks, bool count, cudaStream_t s) {
  if (a.instanced) return count ? cudaErrorInvalidValue : launch_trace_inst(a, blocks, s);
  switch (a.node_format) {
    case kNodeFp32: return launch_fmt<kNodeFp32>(a, blocks, count, s);
    case kNodeFp16: return launch_fmt<kNodeFp16>(a, blocks, count, s);
    case kNodeQ8: return launch_fmt<kNodeQ8>(a, blocks, count, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ags
