// Brute-force render (a test and debugging aid): one thread per ray tests
// every BVH reference of its environment with the render kernel's own ray
// set-up and triangle test, no tree. Culling in the BVH walk is conservative
// and ties are broken the same way, so the two must agree bit for bit; this
// checks the trees on every ray of large scenes, where the FP64 oracle can
// only sample.
#include "trace_kernel.cuh"

namespace ags {
namespace {

// Environment of every leaf-order triangle copy (its input triangle's range
// in the per-environment triangle offsets), keyed for a stable sort that
// groups each environment's copies.
__global__ void k_copy_env(const int32_t* __restrict__ leaf_tri, int32_t R, const int32_t* __restrict__ env_tri,
                           int32_t E, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R) return;
  const int32_t t = leaf_tri[k];
  int32_t lo = 0, hi = E;  // last e with env_tri[e] <= t
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (env_tri[mid] <= t) lo = mid;
    else hi = mid;
  }
  keys[k] = (uint64_t)lo;
  vals[k] = (uint32_t)k;
}

constexpr int kBruteThreads = 256;

__global__ void __launch_bounds__(kBruteThreads) k_brute(const TraceArgs a, const int32_t* __restrict__ env_ref,
                                                         const uint32_t* __restrict__ copies) {
  __shared__ float4 s_frames[kBruteThreads * 3];
  const SensorParams& sen = a.sensor;
  const int64_t per = (int64_t)sen.W * sen.H;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per * a.n) return;
  const int32_t slot = (int32_t)(i / per);
  const int32_t pix = (int32_t)(i - (int64_t)slot * per);
  const int32_t row = pix / sen.W, col = pix - row * sen.W;
  const int32_t env = a.env_ids ? __ldg(a.env_ids + slot) : slot;
  if ((unsigned)env >= (unsigned)a.n_scene_envs) {
    atomicOr(a.status, kStatusBadIndex);
    return;
  }
  const float* P = a.poses + 7 * (int64_t)slot;
  Ray r;
  r.frame = s_frames + 3 * threadIdx.x;
  float R[9], lx, ly, lz;
  if (!make_ray<false>(sen, P, row, col, r, R, lx, ly, lz)) {
    atomicOr(a.status, kStatusBadPose);
    a.out_depth[i] = __int_as_float(0x7fc00000);
    a.out_seg[i] = -1;
    return;
  }
  float t_best = sen.max_range;
  int32_t best_id = 0x7fffffff, best_seg = -1, best_k = -1;
  const int32_t k0 = __ldg(env_ref + env), k1 = __ldg(env_ref + env + 1);
  for (int32_t j = k0; j < k1; ++j) {
    const int32_t k = (int32_t)__ldg(copies + j);
    if (k < a.n_tris) test_triangle<false>(r, a.tris, k, t_best, best_id, best_seg, best_k);
  }
  float v;
  int32_t seg;
  if (best_id != 0x7fffffff) {
    v = t_best;
    seg = best_seg;
    if (v < sen.min_range) {
      if (sen.near_mode == AGS_NEAR_CLAMP) {
        v = sen.min_range;
      } else {
        v = sen.max_range;
        seg = -1;
      }
    }
  } else {
    v = sen.max_range;
    seg = -1;
  }
  a.out_depth[i] = v;
  a.out_seg[i] = seg;
}

// byte offset of the sort's scratch after the keys and values (256-byte aligned)
size_t sort_offset(int32_t R) { return ((size_t)R * 24 + 255) & ~(size_t)255; }

}  // namespace

cudaError_t launch_brute(const TraceArgs& a, const int32_t* env_ref_dev, const int32_t* env_tri_dev,
                         const int32_t* leaf_tri_dev, int32_t E, int32_t R, void* temp, cudaStream_t s) {
  // temp: brute_temp_bytes(R) bytes
  char* p = static_cast<char*>(temp);
  uint64_t* keys = reinterpret_cast<uint64_t*>(p);
  uint64_t* alt_keys = keys + R;
  uint32_t* vals = reinterpret_cast<uint32_t*>(alt_keys + R);
  uint32_t* alt_vals = vals + R;
  void* sort_tmp = p + sort_offset(R);
  cudaError_t e;
  if (R > 0) {
    k_copy_env<<<(R + 255) / 256, 256, 0, s>>>(leaf_tri_dev, R, env_tri_dev, E, keys, vals);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int bits = 1;
    while ((1ll << bits) < E) ++bits;
    if ((e = sort_pairs(keys, vals, alt_keys, alt_vals, R, bits, sort_tmp, s)) != cudaSuccess) return e;
  }
  const int64_t n = (int64_t)a.sensor.W * a.sensor.H * a.n;
  if (n == 0) return cudaSuccess;
  k_brute<<<(unsigned)((n + kBruteThreads - 1) / kBruteThreads), kBruteThreads, 0, s>>>(a, env_ref_dev, vals);
  return cudaGetLastError();
}

size_t brute_temp_bytes(int32_t R) { return sort_offset(R) + sort_temp_bytes(R); }

}  // namespace ags
