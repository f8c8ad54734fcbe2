// Stable LSD radix sort of (uint64 key, uint32 value) pairs and a device-wide
// exclusive scan. Used by the per-environment LBVH build: keys are
// (environment, Morton code) so one global sort orders every environment's
// triangles along its own space-filling curve.
#include "internal.cuh"

namespace ags {

namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kTile = kSortThreads * kSortItems;
constexpr int kWarps = kSortThreads / 32;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Per-tile digit histogram, stored digit-major: hist[d * n_tiles + tile].
__global__ void __launch_bounds__(kSortThreads) k_histogram(const uint64_t* __restrict__ keys, int64_t n,
                                                            int shift, int32_t* __restrict__ hist,
                                                            int32_t n_tiles) {
  __shared__ int32_t cnt[kRadix];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kRadix - 1)], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: items are taken in input order in rounds of kSortThreads;
// within a round, warps in order and lanes in order, so equal digits keep
// their relative order.
__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint64_t* __restrict__ keys_in,
                                                          const uint32_t* __restrict__ vals_in,
                                                          uint64_t* __restrict__ keys_out,
                                                          uint32_t* __restrict__ vals_out, int64_t n,
                                                          int shift, const int32_t* __restrict__ offsets,
                                                          int32_t n_tiles) {
  __shared__ int32_t base_off[kRadix];
  __shared__ int32_t wcnt[kWarps][kRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base_off[tid] = offsets[(int64_t)tid * n_tiles + blockIdx.x];
  for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  const unsigned lt_mask = (1u << lane) - 1u;
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * kSortThreads + tid;
    bool valid = i < n;
    uint64_t key = valid ? keys_in[i] : 0ull;
    uint32_t val = valid ? vals_in[i] : 0u;
    int d = valid ? (int)((key >> shift) & (kRadix - 1)) : kRadix + lane;  // invalid: unique groups
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    // thread tid owns digit tid: exclusive prefix over warps, then advance base
    {
      int acc = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        int c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      // stash the round total in a register until everyone has read offsets
      __syncthreads();
      if (valid) {
        int64_t pos = (int64_t)base_off[d] + wcnt[warp][d] + rank;
        keys_out[pos] = key;
        vals_out[pos] = val;
      }
      __syncthreads();
      base_off[tid] += acc;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- scan
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* warp_sums, int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t s = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  int32_t before = warp > 0 ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  return before + x - v;
}

// Scan each tile of kScanTile items in place (exclusive); write tile sums.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int32_t* __restrict__ data, int64_t n,
                                                             int32_t* __restrict__ tile_sums) {
  __shared__ int32_t warp_sums[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? data[base + k] : 0;
    s += v[k];
  }
  int32_t total;
  int32_t ex = block_exclusive_scan(s, warp_sums, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) data[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int32_t* __restrict__ data, int64_t n, const int32_t* __restrict__ tile_offsets) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  int32_t add = tile_offsets[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) data[i] += add;
}

__global__ void k_scan_total(const int32_t* last_ex, const int32_t* last_val_copy, int32_t* total) {
  *total = *last_ex + *last_val_copy;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

size_t scan_temp_bytes(int64_t n) {
  size_t bytes = 256;  // last value copy
  int64_t m = n > 0 ? n : 1;
  do {
    m = ceil_div(m, kScanTile);
    bytes += ((size_t)m * sizeof(int32_t) + 255) & ~size_t(255);
  } while (m > 1);
  return bytes + 256;
}

cudaError_t exclusive_scan(int32_t* data, int64_t n, int32_t* total_dev, void* temp, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(total_dev, 0, sizeof(int32_t), s);
  char* t = static_cast<char*>(temp);
  int32_t* last_copy = reinterpret_cast<int32_t*>(t);
  t += 256;
  cudaError_t e = cudaMemcpyAsync(last_copy, data + n - 1, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  // levels of tile sums; every level is scanned, down to a single tile
  std::vector<int32_t*> lv_data{data};
  std::vector<int64_t> lv_n{n};
  int64_t tiles;
  do {
    tiles = ceil_div(lv_n.back(), kScanTile);
    int32_t* sums = reinterpret_cast<int32_t*>(t);
    t += ((size_t)tiles * sizeof(int32_t) + 255) & ~size_t(255);
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(lv_data.back(), lv_n.back(), sums);
    lv_data.push_back(sums);
    lv_n.push_back(tiles);
  } while (tiles > 1);
  for (size_t l = lv_data.size() - 1; l-- > 1;) {
    // lv_data[l] scanned (exclusive) including its own tile sums added; add to level l-1
    k_scan_add<<<(unsigned)ceil_div(lv_n[l - 1], kScanTile), kScanThreads, 0, s>>>(lv_data[l - 1], lv_n[l - 1],
                                                                                   lv_data[l]);
  }
  k_scan_total<<<1, 1, 0, s>>>(data + n - 1, last_copy, total_dev);
  return cudaGetLastError();
}

size_t sort_temp_bytes(int64_t n) {
  int64_t tiles = ceil_div(n > 0 ? n : 1, kTile);
  size_t hist = (size_t)tiles * kRadix;
  return ((hist * sizeof(int32_t) + 255) & ~size_t(255)) + scan_temp_bytes((int64_t)hist) + 256;
}

cudaError_t sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* alt_keys, uint32_t* alt_vals, int64_t n,
                       int end_bit, void* temp, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  int32_t tiles = (int32_t)ceil_div(n, kTile);
  int64_t hist_n = (int64_t)tiles * kRadix;
  char* t = static_cast<char*>(temp);
  int32_t* hist = reinterpret_cast<int32_t*>(t);
  t += (hist_n * sizeof(int32_t) + 255) & ~size_t(255);
  int32_t* total = reinterpret_cast<int32_t*>(t);
  t += 256;
  void* scan_tmp = t;
  uint64_t *ki = keys, *ko = alt_keys;
  uint32_t *vi = vals, *vo = alt_vals;
  int passes = 0;
  for (int shift = 0; shift < end_bit; shift += kRadixBits, ++passes) {
    k_histogram<<<tiles, kSortThreads, 0, s>>>(ki, n, shift, hist, tiles);
    cudaError_t e = exclusive_scan(hist, hist_n, total, scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_scatter<<<tiles, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, hist, tiles);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint64_t* tk = ki; ki = ko; ko = tk;
    uint32_t* tv = vi; vi = vo; vo = tv;
  }
  if (passes & 1) {
    cudaError_t e = cudaMemcpyAsync(keys, ki, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(vals, vi, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace ags
