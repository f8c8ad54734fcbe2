// Render-kernel variants with extra work, selected by TraceArgs::extra:
// bit 0 hit channels (face index, barycentrics, normal, sensor-frame point),
// bit 1 stereo shadows, bit 2 a caller's table of sensor-frame directions.
// They use the 8x4 warp tile. Kept apart from trace.cu so the two compile in
// parallel.
#include "trace_kernel.cuh"

namespace ags {
namespace {

template <int kFmt, int kExtra>
void launch_one(const TraceArgs& a, int blocks, cudaStream_t s) {
  k_trace<false, 8, 1, false, kFmt, kExtra><<<blocks, kTraceThreads, 0, s>>>(a);
}

template <int kFmt>
cudaError_t launch_extra_fmt(const TraceArgs& a, int blocks, cudaStream_t s) {
  switch (a.extra) {
    case 1: launch_one<kFmt, 1>(a, blocks, s); break;
    case 2: launch_one<kFmt, 2>(a, blocks, s); break;
    case 3: launch_one<kFmt, 3>(a, blocks, s); break;
    case 4: launch_one<kFmt, 4>(a, blocks, s); break;
    case 5: launch_one<kFmt, 5>(a, blocks, s); break;
    case 6: launch_one<kFmt, 6>(a, blocks, s); break;
    case 7: launch_one<kFmt, 7>(a, blocks, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trace_extra(const TraceArgs& a, int blocks, cudaStream_t s) {
  switch (a.node_format) {
    case kNodeFp32: return launch_extra_fmt<kNodeFp32>(a, blocks, s);
    case kNodeFp16: return launch_extra_fmt<kNodeFp16>(a, blocks, s);
    case kNodeQ8: return launch_extra_fmt<kNodeQ8>(a, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ags
