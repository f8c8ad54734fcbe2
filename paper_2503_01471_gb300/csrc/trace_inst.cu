// The render kernel of two-level scenes (objects with their own BVHs under a
// per-environment BVH over the objects' boxes): 8x4 warp tiles, float32 nodes.
// It reuses the single-level kernel's ray set-up, node test and triangle test
// (trace_kernel.cuh).
#include "trace_kernel.cuh"

namespace ags {

namespace {

// ---------------------------------------------------------------- two-level scenes
// Nearest-hit test of packed triangle k of an object whose triangles start at
// environment-local index tri_base (the index used for ties stays
// environment-local, as in a single-level scene).
__device__ __forceinline__ void test_object_triangle(const Ray& r, const float4* __restrict__ tris, int32_t k,
                                                     int32_t tri_base, float& t_best, int32_t& best_id,
                                                     int32_t& best_seg) {
  const float4 a = __ldg(tris + 3 * (int64_t)k);
  const float4 b = __ldg(tris + 3 * (int64_t)k + 1);
  const float4 c = __ldg(tris + 3 * (int64_t)k + 2);
  const float4 f[3] = {r.frame[0], r.frame[1], r.frame[2]};
  float Ax, Ay, Az, Bx, By, Bz, Cx, Cy, Cz;
  shear(f, a, Ax, Ay, Az);
  shear(f, b, Bx, By, Bz);
  shear(f, c, Cx, Cy, Cz);
  const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  const bool neg = (U < 0.0f) || (V < 0.0f) || (W < 0.0f);
  const bool pos = (U > 0.0f) || (V > 0.0f) || (W > 0.0f);
  if (neg && pos) return;
  const float det = U + V + W;
  if (det == 0.0f) return;
  const float T = __fmaf_rn(U, Az, __fmaf_rn(V, Bz, __fmul_rn(W, Cz)));
  if (T != 0.0f && ((__float_as_uint(T) ^ __float_as_uint(det)) >> 31)) return;
  const float aT = fabsf(T), adet = fabsf(det);
  if (aT > t_best * adet * kCullSlack) return;
  const float t = __fdiv_rn(aT, adet);
  const int32_t id = __float_as_int(b.w) + tri_base;
  if (t < t_best || (t == t_best && id < best_id)) {
    t_best = t;
    best_id = id;
    best_seg = __float_as_int(a.w);
  }
}

// Hit slots of a wide node, nearest first: pushes all but the nearest as
// stack entries {code, entry distance} (the farthest deepest) and returns the
// nearest's code, or -1 when none is left within the cull distance. code(k)
// names slot k's entry. Shared by both levels of a two-level scene.
template <class Code>
__device__ __forceinline__ int32_t order_hits(uint32_t hits, const float* tmins, Code code, float t_best,
                                              int2* stack, int& sp, int* status, bool& failed) {
  const uint32_t key_cull = __float_as_uint(t_best * kCullSlack);
  if (__popc(hits) == 2) {
    // two: the nearer is taken, the farther pushed (keys: entry distance bits, slot in the low 3 bits)
    uint32_t kmin = 0xFFFFFFFFu, kx = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t key = (__float_as_uint(tmins[k]) & ~7u) | (uint32_t)k;
      const bool v = (hits >> k) & 1u;
      kmin = v ? min(kmin, key) : kmin;
      kx ^= v ? key : 0u;
    }
    const uint32_t kfar = kx ^ kmin;
    if ((kfar & ~7u) <= key_cull) {
      if (sp >= kStackSize) {
        atomicOr(status, kStatusStackOverflow);
        failed = true;
        return -1;
      }
      stack[sp++] = make_int2(code((int)(kfar & 7u)), (int32_t)(kfar & ~7u));
    }
    return (kmin & ~7u) <= key_cull ? code((int)(kmin & 7u)) : -1;
  }
  uint32_t keys[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    keys[k] = ((hits >> k) & 1u) ? ((__float_as_uint(tmins[k]) & ~7u) | (uint32_t)k) : 0xFFFFFFFFu;
#define AGS_CSWAP2(i, j)                        \
  {                                             \
    const uint32_t lo_ = min(keys[i], keys[j]); \
    const uint32_t hi_ = max(keys[i], keys[j]); \
    keys[i] = lo_;                              \
    keys[j] = hi_;                              \
  }
  AGS_CSWAP2(0, 1) AGS_CSWAP2(2, 3) AGS_CSWAP2(4, 5) AGS_CSWAP2(6, 7)
  AGS_CSWAP2(0, 2) AGS_CSWAP2(1, 3) AGS_CSWAP2(4, 6) AGS_CSWAP2(5, 7)
  AGS_CSWAP2(1, 2) AGS_CSWAP2(5, 6) AGS_CSWAP2(0, 4) AGS_CSWAP2(3, 7)
  AGS_CSWAP2(1, 5) AGS_CSWAP2(2, 6)
  AGS_CSWAP2(1, 4) AGS_CSWAP2(3, 6)
  AGS_CSWAP2(2, 4) AGS_CSWAP2(3, 5)
  AGS_CSWAP2(3, 4)
#undef AGS_CSWAP2
#pragma unroll
  for (int k = 7; k >= 1; --k) {
    if (keys[k] != 0xFFFFFFFFu && (keys[k] & ~7u) <= key_cull) {
      if (sp >= kStackSize) {
        atomicOr(status, kStatusStackOverflow);
        failed = true;
        return -1;
      }
      stack[sp++] = make_int2(code((int)(keys[k] & 7u)), (int32_t)(keys[k] & ~7u));
    }
  }
  return (keys[0] & ~7u) <= key_cull ? code((int)(keys[0] & 7u)) : -1;
}

// Next entry from the stack above sp0 that is still within the cull distance.
__device__ __forceinline__ int32_t pop_entry(const int2* stack, int& sp, int sp0, float t_best) {
  const float t_pop = t_best * kCullSlack;
  while (sp > sp0) {
    const int2 e = stack[--sp];
    if (__int_as_float(e.y) <= t_pop) return e.x;
  }
  return -1;
}

// The ray r moved into object j's frame: o' = R^T (o - p), d' = R^T d (a
// rigid motion, so distances along the ray are unchanged).
__device__ __forceinline__ void object_ray(const InstanceDev* I, float ox, float oy, float oz, float dx, float dy,
                                           float dz, Ray& r) {
  float rt[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) rt[k] = __ldg(&I->rt[k]);
  const float ax = __fsub_rn(ox, __ldg(&I->p[0])), ay = __fsub_rn(oy, __ldg(&I->p[1])),
              az = __fsub_rn(oz, __ldg(&I->p[2]));
  setup_ray(r, __fmaf_rn(rt[2], az, __fmaf_rn(rt[1], ay, __fmul_rn(rt[0], ax))),
            __fmaf_rn(rt[5], az, __fmaf_rn(rt[4], ay, __fmul_rn(rt[3], ax))),
            __fmaf_rn(rt[8], az, __fmaf_rn(rt[7], ay, __fmul_rn(rt[6], ax))),
            __fmaf_rn(rt[2], dz, __fmaf_rn(rt[1], dy, __fmul_rn(rt[0], dx))),
            __fmaf_rn(rt[5], dz, __fmaf_rn(rt[4], dy, __fmul_rn(rt[3], dx))),
            __fmaf_rn(rt[8], dz, __fmaf_rn(rt[7], dy, __fmul_rn(rt[6], dx))));
}

// The object level: one part of an object (a leaf's triangles, or the subtree
// under a node of the object's BVH) walked with the ray r already in the
// object's frame, on the stack above sp0.
__device__ __forceinline__ void walk_part(const TraceArgs& a, const int4 part, const Ray& r, int32_t tri_base,
                                          float& t_best, int32_t& best_id, int32_t& best_seg, int2* stack, int sp0,
                                          int& visits, bool& failed) {
  if (part.y < 0) {
    if (part.z < 0 || part.w < 1 || part.w > kMaxLeafTris || part.z + part.w > a.obj_n_tris) {
      atomicOr(a.status, kStatusBadIndex);
      failed = true;
      return;
    }
    for (int32_t x = 0; x < part.w; ++x)
      test_object_triangle(r, a.obj_tris, part.z + x, tri_base, t_best, best_id, best_seg);
    return;
  }
  int32_t node = part.y;
  int sp = sp0;
  while (node >= 0) {
    if (++visits > a.max_visits) {
      atomicOr(a.status, kStatusIterationCap);
      failed = true;
      return;
    }
    if (node >= a.obj_n_nodes) {
      atomicOr(a.status, kStatusBadIndex);
      failed = true;
      return;
    }
    int32_t child_base, tri_base_node;
    uint32_t meta_lo, meta_hi, hit_mask;
    float tmins[8];
    test_node<kNodeFp32>(a.obj_nodes, node, r, t_best * kCullSlack, child_base, tri_base_node, meta_lo, meta_hi,
                         tmins, hit_mask);
    const uint32_t b0 = meta_lo & 0xFFu;
    const int ni = (b0 & 0x80u) ? (int)min(b0 & 0xFu, 8u) : 0;
    const uint32_t inner_bits = (1u << ni) - 1u;
    uint32_t leaf_mask = hit_mask & ~inner_bits;
    const uint32_t inner_hits = hit_mask & inner_bits;
    while (leaf_mask) {
      const int k = __ffs(leaf_mask) - 1;
      leaf_mask &= leaf_mask - 1;
      const uint32_t m = ((k < 4 ? meta_lo : meta_hi) >> (8 * (k & 3))) & 0xFFu;
      if (m == kMetaEmpty) continue;
      const int32_t start = tri_base_node + (int32_t)(m >> 2);
      const int32_t cnt = (int32_t)(m & 3u) + 1;
      if (start < 0 || start + cnt > a.obj_n_tris) {
        atomicOr(a.status, kStatusBadIndex);
        failed = true;
        return;
      }
      for (int32_t x = 0; x < cnt; ++x)
        test_object_triangle(r, a.obj_tris, start + x, tri_base, t_best, best_id, best_seg);
    }
    const int n_inner = __popc(inner_hits);
    if (n_inner == 1) {
      node = child_base + (__ffs(inner_hits) - 1);
      continue;
    }
    node = -1;
    if (n_inner > 1)
      node = order_hits(inner_hits, tmins, [&](int k) { return child_base + k; }, t_best, stack, sp, a.status,
                        failed);
    if (failed) return;
    if (node < 0) node = pop_entry(stack, sp, sp0, t_best);
  }
}

// The rays of one warp tile of a two-level scene. The top level (in the
// world frame) holds the environment's object parts, one per leaf slot; its
// walk takes every hit slot, inner node or part, nearest first, so a part
// behind the nearest hit found so far is never entered. Entering a part moves
// the ray into its object's frame (kept while consecutive parts belong to the
// same object) and walks the part. Stack entries: an inner node (>= 0) or
// part q (-2 - q). Nearest hit, ties, clamping and misses as in trace_tile.
__device__ __forceinline__ void trace_tile_inst(const TraceArgs& a, const SensorParams& sen, int32_t env,
                                                int32_t t_in, int32_t slot, int lane, int2* stack, float4* frames) {
  constexpr int kTileW = 8, kTileH = 4;
  const int32_t col = (t_in % sen.tiles_x) * kTileW + (lane % kTileW);
  const int32_t row = (t_in / sen.tiles_x) * kTileH + (lane / kTileW);
  const int32_t W = sen.W, H = sen.H;
  if (col >= W || row >= H) return;
  const float* P = a.poses + 7 * (int64_t)slot;
  const int64_t o = (int64_t)slot * H * W + (int64_t)row * W + col;
  float R[9];
  if (!pose_rotation(P, R)) {
    atomicOr(a.status, kStatusBadPose);
    a.out_depth[o] = __int_as_float(0x7fc00000);
    a.out_seg[o] = -1;
    return;
  }
  const float px = __ldg(P), py = __ldg(P + 1), pz = __ldg(P + 2);
  float lx, ly, lz, dx, dy, dz;
  sensor_dir<false>(sen, row, col, lx, ly, lz);
  rotate(R, lx, ly, lz, dx, dy, dz);
  Ray r;  // the world ray meets only the top level's boxes
  r.frame = nullptr;
  setup_ray<false>(r, px, py, pz, dx, dy, dz);

  float t_best = sen.max_range;
  int32_t best_id = 0x7fffffff, best_seg = -1;
  int32_t e = __ldg(a.env_root + env);
  const int32_t j0 = __ldg(a.env_sub + env), j1 = __ldg(a.env_sub + env + 1);
  Ray ro;                       // the ray in the frame of object cur_j
  ro.frame = frames;
  int32_t cur_j = -1, tri_base = 0;
  int sp = 0, visits = 0;
  bool failed = false;
  while (e != -1) {
    if (++visits > a.max_visits) {
      atomicOr(a.status, kStatusIterationCap);
      failed = true;
      break;
    }
    if (e < -1) {
      // a part: its object, then its node or leaf
      const int32_t q = -2 - e;
      if (q >= a.n_tris) {
        atomicOr(a.status, kStatusBadIndex);
        failed = true;
        break;
      }
      const int4 part = __ldg(a.parts + q);
      const int32_t j = part.x;
      if (j < j0 || j >= j1 || j >= a.n_inst) {
        atomicOr(a.status, kStatusBadIndex);
        failed = true;
        break;
      }
      if (j != cur_j) {
        object_ray(a.inst + j, px, py, pz, dx, dy, dz, ro);
        tri_base = __ldg(&a.inst[j].tri_base);
        cur_j = j;
      }
      walk_part(a, part, ro, tri_base, t_best, best_id, best_seg, stack, sp, visits, failed);
      if (failed) break;
      e = pop_entry(stack, sp, 0, t_best);
      continue;
    }
    if (e >= a.n_nodes) {
      atomicOr(a.status, kStatusBadIndex);
      failed = true;
      break;
    }
    int32_t child_base, leaf_base;
    uint32_t meta_lo, meta_hi, hit_mask;
    float tmins[8];
    test_node<kNodeFp32>(a.nodes, e, r, t_best * kCullSlack, child_base, leaf_base, meta_lo, meta_hi, tmins,
                         hit_mask);
    const uint32_t b0 = meta_lo & 0xFFu;
    const int ni = (b0 & 0x80u) ? (int)min(b0 & 0xFu, 8u) : 0;
    // a leaf slot holds one part (the top level is built with one reference per leaf)
    uint32_t leaf_mask = hit_mask & ~((1u << ni) - 1u);
    while (leaf_mask) {
      const int k = __ffs(leaf_mask) - 1;
      leaf_mask &= leaf_mask - 1;
      const uint32_t m = ((k < 4 ? meta_lo : meta_hi) >> (8 * (k & 3))) & 0xFFu;
      if (m == kMetaEmpty) {
        hit_mask &= ~(1u << k);
      } else if ((m & 3u) != 0u) {
        atomicOr(a.status, kStatusBadIndex);
        failed = true;
      }
    }
    if (failed) break;
    auto code = [&](int k) {
      return k < ni ? child_base + k
                    : -2 - (leaf_base + (int32_t)((((k < 4 ? meta_lo : meta_hi) >> (8 * (k & 3))) & 0xFFu) >> 2));
    };
    if (__popc(hit_mask) == 1) {
      e = code(__ffs(hit_mask) - 1);
      continue;
    }
    e = -1;
    if (hit_mask) e = order_hits(hit_mask, tmins, code, t_best, stack, sp, a.status, failed);
    if (failed) break;
    if (e == -1) e = pop_entry(stack, sp, 0, t_best);
  }

  float v;
  int32_t seg;
  if (failed) {
    v = __int_as_float(0x7fc00000);
    seg = -1;
  } else if (best_id != 0x7fffffff) {
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
  a.out_depth[o] = v;
  a.out_seg[o] = seg;
}

// two levels hold two rays; 7 resident blocks per SM, as for k_trace (measured: 10185 Mrays/s on 1024 rooms
// against 9917 with 6 blocks and 9575 with 5, the extra spills costing less than the occupancy gained)
__global__ void __launch_bounds__(kTraceThreads, 7) k_trace_inst(const TraceArgs a) {
  const int lane = threadIdx.x & 31;
  int2 stack[kStackSize];
  // each thread's slot for the triangle-test constants of its ray in an object's frame
  __shared__ float4 s_frames[kTraceThreads * 3];
  float4* frames = s_frames + 3 * threadIdx.x;
  while (true) {
    unsigned int tile = 0;
    if (lane == 0) tile = atomicAdd(a.tile_counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if ((int64_t)tile >= a.total_tiles) break;
    const int32_t slot = (int32_t)(tile / (unsigned)a.sensor.tiles_per_env);
    const int32_t t_in = (int32_t)(tile - (unsigned)slot * (unsigned)a.sensor.tiles_per_env);
    const int32_t env = a.env_ids ? __ldg(a.env_ids + slot) : slot;
    if ((unsigned)env >= (unsigned)a.n_scene_envs) {
      if (lane == 0) atomicOr(a.status, kStatusBadIndex);
      continue;
    }
    trace_tile_inst(a, a.sensor, env, t_in, slot, lane, stack, frames);
  }
}

}  // namespace

cudaError_t launch_trace_inst(const TraceArgs& a, int blocks, cudaStream_t s) {
  if (a.log2_tile_w != 3 || a.rays_per_lane != 1 || a.node_format != kNodeFp32 || a.slots || a.extra)
    return cudaErrorInvalidValue;
  k_trace_inst<<<blocks, kTraceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ags
