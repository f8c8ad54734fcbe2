// Batched ray casting (Sec. III-D.1: "individual rays are cast outwards
// per-pixel to evaluate intersection with M_{i,t}"; range vs depth): one
// persistent launch over every environment's rays. Each warp repeatedly takes
// an 8x4 tile of pixels (env-major order, so one environment's BVH stays hot
// in L2 while all SMs work on it), generates the rays in registers, walks the
// environment's 8-wide BVH with a per-thread stack, tests leaf triangles with
// a watertight float32 test and writes depth/range and segment ID.
#include "internal.cuh"

namespace ags {

namespace {

constexpr int kTraceThreads = 128;
constexpr int kStackSize = 64;
constexpr int kTileW = 8, kTileH = 4;
// Box culling is made conservative against float32 rounding: the slab exit
// is scaled up by (1 + 2 gamma_3) and the current nearest hit by (1 + 2^-12),
// so a box holding the eventual nearest triangle is never skipped.
constexpr float kSlabSlack = 1.0f + 4.0f * 5.96046448e-8f;
constexpr float kCullSlack = 1.0f + 2.44140625e-4f;

struct Ray {
  float ox, oy, oz;
  float dx, dy, dz;
  float ix, iy, iz;
  // watertight test: permuted axes and shear constants
  int kx, ky, kz;
  float Sx, Sy, Sz;
  float okx, oky, okz;
};

__device__ __forceinline__ float nonzero(float d) {
  // an exactly-zero direction component is replaced by a tiny one of the same
  // sign for both the box and the triangle test, keeping them consistent
  return fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d;
}

__device__ __forceinline__ float sel3(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

__device__ __forceinline__ void setup_ray(Ray& r) {
  r.dx = nonzero(r.dx);
  r.dy = nonzero(r.dy);
  r.dz = nonzero(r.dz);
  r.ix = 1.0f / r.dx;
  r.iy = 1.0f / r.dy;
  r.iz = 1.0f / r.dz;
  float ax = fabsf(r.dx), ay = fabsf(r.dy), az = fabsf(r.dz);
  int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  float dkz = sel3(r.dx, r.dy, r.dz, kz);
  if (dkz < 0.0f) {  // keep the winding so the edge tests stay consistent
    int t = kx;
    kx = ky;
    ky = t;
  }
  r.kx = kx;
  r.ky = ky;
  r.kz = kz;
  r.Sx = sel3(r.dx, r.dy, r.dz, kx) / dkz;
  r.Sy = sel3(r.dx, r.dy, r.dz, ky) / dkz;
  r.Sz = 1.0f / dkz;
  r.okx = sel3(r.ox, r.oy, r.oz, kx);
  r.oky = sel3(r.ox, r.oy, r.oz, ky);
  r.okz = sel3(r.ox, r.oy, r.oz, kz);
}

// Watertight ray/triangle test (Woop, Benthin, Wald 2013), two-sided with
// closed edges. Each edge function is an explicitly rounded difference of two
// rounded products, so a shared edge gives exactly opposite values in its two
// triangles and no ray slips between them.
__device__ __forceinline__ void test_triangle(const Ray& r, const float4* __restrict__ tris, int32_t k,
                                              float& t_best, int32_t& best_id, int32_t& best_seg) {
  const float4 a = __ldg(tris + 3 * (int64_t)k);
  const float4 b = __ldg(tris + 3 * (int64_t)k + 1);
  const float4 c = __ldg(tris + 3 * (int64_t)k + 2);
  float ax = __fsub_rn(sel3(a.x, a.y, a.z, r.kx), r.okx);
  float ay = __fsub_rn(sel3(a.x, a.y, a.z, r.ky), r.oky);
  float az = __fsub_rn(sel3(a.x, a.y, a.z, r.kz), r.okz);
  float bx = __fsub_rn(sel3(b.x, b.y, b.z, r.kx), r.okx);
  float by = __fsub_rn(sel3(b.x, b.y, b.z, r.ky), r.oky);
  float bz = __fsub_rn(sel3(b.x, b.y, b.z, r.kz), r.okz);
  float cx = __fsub_rn(sel3(c.x, c.y, c.z, r.kx), r.okx);
  float cy = __fsub_rn(sel3(c.x, c.y, c.z, r.ky), r.oky);
  float cz = __fsub_rn(sel3(c.x, c.y, c.z, r.kz), r.okz);
  const float Ax = __fmaf_rn(-r.Sx, az, ax), Ay = __fmaf_rn(-r.Sy, az, ay);
  const float Bx = __fmaf_rn(-r.Sx, bz, bx), By = __fmaf_rn(-r.Sy, bz, by);
  const float Cx = __fmaf_rn(-r.Sx, cz, cx), Cy = __fmaf_rn(-r.Sy, cz, cy);
  const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  const bool neg = (U < 0.0f) || (V < 0.0f) || (W < 0.0f);
  const bool pos = (U > 0.0f) || (V > 0.0f) || (W > 0.0f);
  if (neg && pos) return;
  const float det = U + V + W;
  if (det == 0.0f) return;
  const float T = __fmaf_rn(U, r.Sz * az, __fmaf_rn(V, r.Sz * bz, __fmul_rn(W, r.Sz * cz)));
  // cheap reject before the division: |t| beyond the current best (with slack)
  const float aT = fabsf(T), adet = fabsf(det);
  if (T != 0.0f && ((__float_as_uint(T) ^ __float_as_uint(det)) >> 31)) return;  // t < 0
  if (aT > t_best * adet * kCullSlack) return;
  const float t = __fdiv_rn(aT, adet);
  const int32_t id = __float_as_int(b.w);
  if (t < t_best || (t == t_best && id < best_id)) {
    t_best = t;
    best_id = id;
    best_seg = __float_as_int(a.w);
  }
}

template <bool kCount>
__global__ void __launch_bounds__(kTraceThreads) k_trace(const TraceArgs a) {
  const int lane = threadIdx.x & 31;
  int32_t* __restrict__ status = a.status;
  int2 stack[kStackSize];
  unsigned long long n_nodes = 0, n_tris = 0, n_rays = 0;

  while (true) {
    unsigned int tile = 0;
    if (lane == 0) tile = atomicAdd(a.tile_counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if ((int64_t)tile >= a.total_tiles) break;
    const int32_t slot = (int32_t)(tile / (unsigned)a.tiles_per_env);
    const int32_t t_in = (int32_t)(tile - (unsigned)slot * (unsigned)a.tiles_per_env);
    const int32_t env = a.env_ids ? __ldg(a.env_ids + slot) : slot;
    if ((unsigned)env >= (unsigned)a.n_scene_envs) {
      if (lane == 0) atomicOr(a.status, kStatusBadIndex);
      continue;
    }
    const int32_t col = (t_in % a.tiles_x) * kTileW + (lane & (kTileW - 1));
    const int32_t row = (t_in / a.tiles_x) * kTileH + (lane >> 3);
    if (col >= a.W || row >= a.H) continue;

    // ---- a3: ray generation from the sensor pose (p, q)
    const float* P = a.poses + 7 * (int64_t)slot;
    const float px = __ldg(P), py = __ldg(P + 1), pz = __ldg(P + 2);
    const float qx = __ldg(P + 3), qy = __ldg(P + 4), qz = __ldg(P + 5), qw = __ldg(P + 6);
    const float n2 = qx * qx + qy * qy + qz * qz + qw * qw;
    if (!(n2 >= 1e-30f) || !isfinite(n2) || !isfinite(px + py + pz)) {
      // a pose the method cannot use: flag it and report NaN for this ray
      atomicOr(status, kStatusBadPose);
      if (!kCount) {
        const int64_t o = ((int64_t)slot * a.H + row) * a.W + col;
        a.out_depth[o] = __int_as_float(0x7fc00000);
        a.out_seg[o] = -1;
      }
      continue;
    }
    const float s = 2.0f / n2;
    const float R00 = 1.0f - s * (qy * qy + qz * qz), R01 = s * (qx * qy - qz * qw), R02 = s * (qx * qz + qy * qw);
    const float R10 = s * (qx * qy + qz * qw), R11 = 1.0f - s * (qx * qx + qz * qz), R12 = s * (qy * qz - qx * qw);
    const float R20 = s * (qx * qz - qy * qw), R21 = s * (qy * qz + qx * qw), R22 = 1.0f - s * (qx * qx + qy * qy);
    float lx, ly, lz;
    if (a.type == AGS_PINHOLE) {
      // unnormalised (1, a, b): the distance along it is the depth itself
      lx = 1.0f;
      ly = (0.5f * (float)a.W - ((float)col + 0.5f)) * a.inv_f;
      lz = (0.5f * (float)a.H - ((float)row + 0.5f)) * a.inv_f;
    } else {
      float sin_el, cos_el, sin_az, cos_az;
      sincosf(a.vmax - (float)row * a.dv, &sin_el, &cos_el);
      sincosf(a.hfov * ((float)col / (float)a.W), &sin_az, &cos_az);
      lx = cos_el * cos_az;
      ly = cos_el * sin_az;
      lz = sin_el;
    }
    Ray r;
    r.ox = px;
    r.oy = py;
    r.oz = pz;
    r.dx = R00 * lx + R01 * ly + R02 * lz;
    r.dy = R10 * lx + R11 * ly + R12 * lz;
    r.dz = R20 * lx + R21 * ly + R22 * lz;
    setup_ray(r);

    // ---- a4-a6: traversal, triangle tests, nearest hit
    float t_best = a.max_range;  // camera: depth limit; LiDAR: range limit (unit direction)
    int32_t best_id = 0x7fffffff, best_seg = -1;
    int32_t node = __ldg(a.env_root + env);
    int sp = 0, visits = 0;
    bool failed = false;
    while (node >= 0) {
      if (++visits > a.max_visits) {
        atomicOr(status, kStatusIterationCap);
        failed = true;
        break;
      }
      if (node >= a.n_nodes) {
        atomicOr(status, kStatusBadIndex);
        failed = true;
        break;
      }
      if (kCount) ++n_nodes;
      const float4* np = reinterpret_cast<const float4*>(a.nodes + node);
      const float4 h = __ldg(np);
      const int32_t child_base = __float_as_int(h.x), tri_base = __float_as_int(h.y);
      const uint32_t meta_lo = __float_as_uint(h.z), meta_hi = __float_as_uint(h.w);
      const float t_cull = t_best * kCullSlack;
      uint32_t keys[8];
      uint32_t leaf_mask = 0;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const float4 lx4 = __ldg(np + 1 + half), hx4 = __ldg(np + 3 + half);
        const float4 ly4 = __ldg(np + 5 + half), hy4 = __ldg(np + 7 + half);
        const float4 lz4 = __ldg(np + 9 + half), hz4 = __ldg(np + 11 + half);
        const float lxs[4] = {lx4.x, lx4.y, lx4.z, lx4.w}, hxs[4] = {hx4.x, hx4.y, hx4.z, hx4.w};
        const float lys[4] = {ly4.x, ly4.y, ly4.z, ly4.w}, hys[4] = {hy4.x, hy4.y, hy4.z, hy4.w};
        const float lzs[4] = {lz4.x, lz4.y, lz4.z, lz4.w}, hzs[4] = {hz4.x, hz4.y, hz4.z, hz4.w};
        const uint32_t meta = half ? meta_hi : meta_lo;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k = 4 * half + q;
          const float tx0 = __fmul_rn(__fsub_rn(lxs[q], r.ox), r.ix), tx1 = __fmul_rn(__fsub_rn(hxs[q], r.ox), r.ix);
          const float ty0 = __fmul_rn(__fsub_rn(lys[q], r.oy), r.iy), ty1 = __fmul_rn(__fsub_rn(hys[q], r.oy), r.iy);
          const float tz0 = __fmul_rn(__fsub_rn(lzs[q], r.oz), r.iz), tz1 = __fmul_rn(__fsub_rn(hzs[q], r.oz), r.iz);
          const float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
          const float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1)) * kSlabSlack;
          const bool hit = tmin <= fminf(tmax, t_cull);
          const uint32_t m = (meta >> (8 * q)) & 0xFFu;
          const bool inner = (m & 0xF8u) == 0x80u;  // 0x80..0x87; 0xFF is an empty slot
          keys[k] = (hit && inner) ? ((__float_as_uint(tmin) & ~7u) | (m & 7u)) : 0xFFFFFFFFu;
          if (hit && !inner) leaf_mask |= 1u << k;
        }
      }
      // leaves of this node first: they tighten t_best before descending
      while (leaf_mask) {
        const int k = __ffs(leaf_mask) - 1;
        leaf_mask &= leaf_mask - 1;
        const uint32_t m = ((k < 4 ? meta_lo : meta_hi) >> (8 * (k & 3))) & 0xFFu;
        const int32_t start = tri_base + (int32_t)(m >> 2);
        const int32_t cnt = (int32_t)(m & 3u) + 1;
        if (start < 0 || start + cnt > a.n_tris) {
          atomicOr(status, kStatusBadIndex);
          failed = true;
          break;
        }
        for (int32_t x = 0; x < cnt; ++x) test_triangle(r, a.tris, start + x, t_best, best_id, best_seg);
        if (kCount) n_tris += cnt;
      }
      if (failed) break;
      // inner children, nearest first (sorting network on packed keys)
#define AGS_CSWAP(i, j)                      \
  {                                          \
    const uint32_t lo_ = min(keys[i], keys[j]); \
    const uint32_t hi_ = max(keys[i], keys[j]); \
    keys[i] = lo_;                           \
    keys[j] = hi_;                           \
  }
      AGS_CSWAP(0, 1) AGS_CSWAP(2, 3) AGS_CSWAP(4, 5) AGS_CSWAP(6, 7)
      AGS_CSWAP(0, 2) AGS_CSWAP(1, 3) AGS_CSWAP(4, 6) AGS_CSWAP(5, 7)
      AGS_CSWAP(1, 2) AGS_CSWAP(5, 6) AGS_CSWAP(0, 4) AGS_CSWAP(3, 7)
      AGS_CSWAP(1, 5) AGS_CSWAP(2, 6)
      AGS_CSWAP(1, 4) AGS_CSWAP(3, 6)
      AGS_CSWAP(2, 4) AGS_CSWAP(3, 5)
      AGS_CSWAP(3, 4)
#undef AGS_CSWAP
      const uint32_t key_cull = __float_as_uint(t_best * kCullSlack);
#pragma unroll
      for (int k = 7; k >= 1; --k) {
        if (keys[k] != 0xFFFFFFFFu && (keys[k] & ~7u) <= key_cull) {
          if (sp >= kStackSize) {
            atomicOr(status, kStatusStackOverflow);
            failed = true;
          } else {
            stack[sp++] = make_int2(child_base + (int32_t)(keys[k] & 7u), (int32_t)(keys[k] & ~7u));
          }
        }
      }
      if (failed) break;
      if (keys[0] != 0xFFFFFFFFu && (keys[0] & ~7u) <= key_cull) {
        node = child_base + (int32_t)(keys[0] & 7u);
        continue;
      }
      node = -1;
      const float t_pop = t_best * kCullSlack;
      while (sp > 0) {
        const int2 e = stack[--sp];
        if (__int_as_float(e.y) <= t_pop) {
          node = e.x;
          break;
        }
      }
    }

    if (kCount) {
      ++n_rays;
      continue;
    }
    float v;
    int32_t seg;
    if (failed) {
      v = __int_as_float(0x7fc00000);
      seg = -1;
    } else if (best_id != 0x7fffffff) {
      v = t_best;
      seg = best_seg;
      if (v < a.min_range) {
        if (a.near_mode == AGS_NEAR_CLAMP) {
          v = a.min_range;
        } else {
          v = a.max_range;
          seg = -1;
        }
      }
    } else {
      v = a.max_range;
      seg = -1;
    }
    const int64_t o = ((int64_t)slot * a.H + row) * a.W + col;
    a.out_depth[o] = v;
    a.out_seg[o] = seg;
  }
  if (kCount) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_nodes += __shfl_xor_sync(0xffffffffu, n_nodes, o);
      n_tris += __shfl_xor_sync(0xffffffffu, n_tris, o);
      n_rays += __shfl_xor_sync(0xffffffffu, n_rays, o);
    }
    if (lane == 0) {
      atomicAdd(a.counts, n_rays);
      atomicAdd(a.counts + 1, n_nodes);
      atomicAdd(a.counts + 2, n_tris);
    }
  }
}

}  // namespace

int trace_blocks_per_sm(bool count) {
  int n = 0;
  cudaError_t e = count ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<true>, kTraceThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<false>, kTraceThreads, 0);
  return (e == cudaSuccess && n > 0) ? n : 1;
}

cudaError_t launch_trace(const TraceArgs& a, int blocks, bool count, cudaStream_t s) {
  if (count) k_trace<true><<<blocks, kTraceThreads, 0, s>>>(a);
  else k_trace<false><<<blocks, kTraceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ags
