// Scene build: object-to-world transform (Sec. III-D.1, M_{i,t} from the
// per-object transforms T_{j,t}) and one BVH per environment's meshes M_{i,t}
// (Sec. III-D.1), as an LBVH (Morton codes,
// radix sort, Karras-style radix tree, bottom-up bounds refit) collapsed into
// 8-wide nodes. All environments are built together, in one pass per stage.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_fp16.h>

#include "internal.cuh"

namespace ags {

namespace {


// ---------------------------------------------------------------- float-float
// Transform arithmetic in unevaluated float pairs (hi + lo) built from
// error-free products (fma) and sums, so the float32 world vertex is within
// one unit in the last place of the exact value without any double math.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_fast_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_fast_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_sum(p, e);
}
__device__ __forceinline__ ff ff_of(float a) { return {a, 0.0f}; }
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  ff r = ff_add(a, ff_neg(ff_mul(ff_of(q1), b)));
  float q2 = __fdiv_rn(r.hi, b.hi);
  return ff_fast_sum(q1, q2);
}

// Rotation of the (not necessarily unit) quaternion q: R = I + s K with
// s = 2 / |q|^2, so no square root is needed.
__global__ void k_submesh_rotations(const float* __restrict__ poses, int32_t J, float* __restrict__ rot_ff) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  const float* P = poses + 7 * (int64_t)j;
  ff x = ff_of(P[3]), y = ff_of(P[4]), z = ff_of(P[5]), w = ff_of(P[6]);
  ff xx = ff_mul(x, x), yy = ff_mul(y, y), zz = ff_mul(z, z), ww = ff_mul(w, w);
  ff n2 = ff_add(ff_add(xx, yy), ff_add(zz, ww));
  ff s = ff_div(ff_of(2.0f), n2);
  ff xy = ff_mul(x, y), xz = ff_mul(x, z), yz = ff_mul(y, z);
  ff xw = ff_mul(x, w), yw = ff_mul(y, w), zw = ff_mul(z, w);
  ff one = ff_of(1.0f);
  ff R[9];
  R[0] = ff_add(one, ff_neg(ff_mul(s, ff_add(yy, zz))));
  R[1] = ff_mul(s, ff_add(xy, ff_neg(zw)));
  R[2] = ff_mul(s, ff_add(xz, yw));
  R[3] = ff_mul(s, ff_add(xy, zw));
  R[4] = ff_add(one, ff_neg(ff_mul(s, ff_add(xx, zz))));
  R[5] = ff_mul(s, ff_add(yz, ff_neg(xw)));
  R[6] = ff_mul(s, ff_add(xz, ff_neg(yw)));
  R[7] = ff_mul(s, ff_add(yz, xw));
  R[8] = ff_add(one, ff_neg(ff_mul(s, ff_add(xx, yy))));
  float* o = rot_ff + 18 * (int64_t)j;
  for (int k = 0; k < 9; ++k) {
    o[2 * k] = R[k].hi;
    o[2 * k + 1] = R[k].lo;
  }
}

__device__ __forceinline__ int32_t upper_bound_i32(const int32_t* a, int32_t n, int32_t x) {
  // first index k in [0, n) with a[k] > x  (a sorted ascending)
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// a1: v' = R(q_j) v + p_j for every vertex of sub-mesh j.
__global__ void k_transform_vertices(const float* __restrict__ base, int32_t V, const int32_t* __restrict__ sub_vert_off,
                                     int32_t J, const float* __restrict__ rot_ff, const float* __restrict__ poses,
                                     float4* __restrict__ world) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  int32_t j = upper_bound_i32(sub_vert_off + 1, J, v);  // sub_vert_off[j] <= v < sub_vert_off[j+1]
  const float* r = rot_ff + 18 * (int64_t)j;
  const float* P = poses + 7 * (int64_t)j;
  ff b[3] = {ff_of(base[3 * (int64_t)v]), ff_of(base[3 * (int64_t)v + 1]), ff_of(base[3 * (int64_t)v + 2])};
  float out[3];
#pragma unroll
  for (int row = 0; row < 3; ++row) {
    ff acc = ff_of(P[row]);
    acc = ff_add(acc, ff_mul({r[6 * row + 0], r[6 * row + 1]}, b[0]));
    acc = ff_add(acc, ff_mul({r[6 * row + 2], r[6 * row + 3]}, b[1]));
    acc = ff_add(acc, ff_mul({r[6 * row + 4], r[6 * row + 5]}, b[2]));
    out[row] = __fadd_rn(acc.hi, acc.lo);
  }
  world[v] = make_float4(out[0], out[1], out[2], 0.0f);
}

// Packed triangles in input order; also the environment of each triangle.
__global__ void k_pack_triangles(const int32_t* __restrict__ vidx, int32_t F, const float4* __restrict__ world,
                                 const int32_t* __restrict__ sub_tri_off, int32_t J,
                                 const int32_t* __restrict__ sub_seg, const int32_t* __restrict__ sub_env,
                                 const int32_t* __restrict__ env_tri_off, float4* __restrict__ packed,
                                 int32_t* __restrict__ tri_env) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= F) return;
  int32_t j = upper_bound_i32(sub_tri_off + 1, J, t);
  int32_t e = sub_env[j];
  float4 a = world[vidx[3 * (int64_t)t]];
  float4 b = world[vidx[3 * (int64_t)t + 1]];
  float4 c = world[vidx[3 * (int64_t)t + 2]];
  a.w = __int_as_float(sub_seg[j]);
  b.w = __int_as_float(t - env_tri_off[e]);
  c.w = 0.0f;
  packed[3 * (int64_t)t] = a;
  packed[3 * (int64_t)t + 1] = b;
  packed[3 * (int64_t)t + 2] = c;
  tri_env[t] = e;
}

// order-preserving float <-> int mapping for atomic min/max
__device__ __forceinline__ int32_t f2ord(float f) {
  int32_t i = __float_as_int(f);
  return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float ord2f(int32_t i) { return __int_as_float(i >= 0 ? i : (i ^ 0x7FFFFFFF)); }

__global__ void k_init_bounds(int32_t* b, int32_t E) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int k = 0; k < 3; ++k) {
    b[6 * e + k] = 0x7FFFFFFF;
    b[6 * e + 3 + k] = (int32_t)0x80000000;
  }
}


__device__ __forceinline__ float3 box_center(const Box& b) {
  return make_float3(0.5f * (b.lox + b.hix), 0.5f * (b.loy + b.hiy), 0.5f * (b.loz + b.hiz));
}

// per-environment bounds of reference-box centres (warp-aggregated atomics
// when the whole warp belongs to one environment, per-lane atomics otherwise)
__global__ void k_env_bounds(const Box* __restrict__ boxes, const int32_t* __restrict__ env_of, int32_t n,
                             int32_t* __restrict__ bounds) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = t < n;
  int32_t e = valid ? env_of[t] : -1;
  float3 c = valid ? box_center(boxes[t]) : make_float3(0, 0, 0);
  int32_t v[6] = {f2ord(c.x), f2ord(c.y), f2ord(c.z), f2ord(c.x), f2ord(c.y), f2ord(c.z)};
  unsigned peers = __match_any_sync(0xffffffffu, e);
  if (peers == 0xffffffffu) {  // uniform branch: every lane sees the same mask
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      int32_t x = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        int32_t y = __shfl_xor_sync(0xffffffffu, x, o);
        x = (k < 3) ? min(x, y) : max(x, y);
      }
      v[k] = x;
    }
    if (!valid || (threadIdx.x & 31) != 0) return;
  } else if (!valid) {
    return;
  }
  int32_t* b = bounds + 6 * (int64_t)e;
  for (int k = 0; k < 3; ++k) atomicMin(b + k, v[k]);
  for (int k = 3; k < 6; ++k) atomicMax(b + k, v[k]);
}

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
  // bits of x (up to 21) moved to every third position
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__global__ void k_morton(const Box* __restrict__ boxes, const int32_t* __restrict__ env_of, int32_t n,
                         const int32_t* __restrict__ bounds, int bits, uint64_t* __restrict__ keys,
                         uint32_t* __restrict__ vals) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int32_t e = env_of[t];
  const int32_t* b = bounds + 6 * (int64_t)e;
  float3 c = box_center(boxes[t]);
  float cc[3] = {c.x, c.y, c.z};
  uint64_t q[3];
  const float scale = (float)(1u << bits);
  for (int k = 0; k < 3; ++k) {
    float lo = ord2f(b[k]), hi = ord2f(b[3 + k]);
    float ext = hi - lo;
    float u = ext > 0.0f ? (cc[k] - lo) / ext : 0.0f;
    float sc = fminf(fmaxf(u * scale, 0.0f), scale - 1.0f);
    q[k] = (uint64_t)sc;
  }
  uint64_t m = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
  keys[t] = ((uint64_t)e << (3 * bits)) | m;
  vals[t] = (uint32_t)t;
}

__device__ __forceinline__ Box tri_box(const float4* packed, int64_t t) {
  float4 a = packed[3 * t], b = packed[3 * t + 1], c = packed[3 * t + 2];
  Box x;
  x.lox = fminf(a.x, fminf(b.x, c.x));
  x.loy = fminf(a.y, fminf(b.y, c.y));
  x.loz = fminf(a.z, fminf(b.z, c.z));
  x.hix = fmaxf(a.x, fmaxf(b.x, c.x));
  x.hiy = fmaxf(a.y, fmaxf(b.y, c.y));
  x.hiz = fmaxf(a.z, fmaxf(b.z, c.z));
  return x;
}

__global__ void k_tri_boxes(const float4* __restrict__ packed, int32_t F, Box* __restrict__ out) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < F) out[t] = tri_box(packed, t);
}

// ---------------------------------------------------------------- reference splitting
// A triangle much larger than its environment's cell size gets several BVH
// references: its box is cut into a grid of up to 8 cells per axis (64 in
// all) and each cell that the triangle reaches becomes a reference whose box
// is the triangle clipped to that cell. All references point at the same
// packed triangle, so ray results do not change; the boxes are tighter, so
// traversal enters fewer nodes. Clipped boxes are widened by 2^-19 of the
// coordinate magnitude (beyond the clipping's rounding) and cut back to the
// triangle's exact box, so together they always cover the whole triangle.
constexpr int kSplitMaxPerAxis = 8;
constexpr int kDefaultSplitCells = 16;  // cells across an environment's largest extent
constexpr int kSplitMaxRefs = 64;

struct SplitGrid {
  int n[3];
  float lo[3], hi[3];
};

__device__ __forceinline__ SplitGrid split_grid(const Box& tb, float cell, int max_refs) {
  SplitGrid g;
  g.lo[0] = tb.lox; g.lo[1] = tb.loy; g.lo[2] = tb.loz;
  g.hi[0] = tb.hix; g.hi[1] = tb.hiy; g.hi[2] = tb.hiz;
  for (int a = 0; a < 3; ++a) {
    float ext = g.hi[a] - g.lo[a];
    int k = 1;
    if (cell > 0.0f && ext > cell) k = (int)fminf(ceilf(ext / cell), (float)kSplitMaxPerAxis);
    g.n[a] = max(k, 1);
  }
  while (g.n[0] * g.n[1] * g.n[2] > max_refs) {
    int a = (g.n[0] >= g.n[1] && g.n[0] >= g.n[2]) ? 0 : (g.n[1] >= g.n[2] ? 1 : 2);
    g.n[a] = (g.n[a] + 1) / 2;
  }
  return g;
}

__device__ __forceinline__ float grid_bound(const SplitGrid& g, int a, int i) {
  if (i <= 0) return g.lo[a];
  if (i >= g.n[a]) return g.hi[a];
  return g.lo[a] + (g.hi[a] - g.lo[a]) * ((float)i / (float)g.n[a]);
}

// Clip triangle (a, b, c) to the cell [lo, hi] (Sutherland-Hodgman against
// its six planes); false if nothing is left, else the clipped polygon's box
// and the range of its vertices' barycentric weights (u of b, v of c).
__device__ bool clip_to_cell(const float4& a, const float4& b, const float4& c, const float lo[3],
                             const float hi[3], Box& out, float bary[4]) {
  float P[9][3], Q[9][3];
  P[0][0] = a.x; P[0][1] = a.y; P[0][2] = a.z;
  P[1][0] = b.x; P[1][1] = b.y; P[1][2] = b.z;
  P[2][0] = c.x; P[2][1] = c.y; P[2][2] = c.z;
  int n = 3;
  for (int plane = 0; plane < 6; ++plane) {
    const int ax = plane >> 1;
    const bool upper = plane & 1;
    const float bound = upper ? hi[ax] : lo[ax];
    int m = 0;
    for (int i = 0; i < n; ++i) {
      const float* cur = P[i];
      const float* nxt = P[(i + 1) % n];
      const float dc = upper ? bound - cur[ax] : cur[ax] - bound;
      const float dn = upper ? bound - nxt[ax] : nxt[ax] - bound;
      if (dc >= 0.0f && m < 9) {
        Q[m][0] = cur[0]; Q[m][1] = cur[1]; Q[m][2] = cur[2];
        ++m;
      }
      if (((dc > 0.0f && dn < 0.0f) || (dc < 0.0f && dn > 0.0f)) && m < 9) {
        const float t = dc / (dc - dn);
        for (int k = 0; k < 3; ++k) Q[m][k] = cur[k] + t * (nxt[k] - cur[k]);
        Q[m][ax] = bound;
        ++m;
      }
    }
    n = m;
    if (n == 0) return false;
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) P[i][k] = Q[i][k];
  }
  Box bx = {P[0][0], P[0][1], P[0][2], P[0][0], P[0][1], P[0][2]};
  for (int i = 1; i < n; ++i) {
    bx.lox = fminf(bx.lox, P[i][0]); bx.hix = fmaxf(bx.hix, P[i][0]);
    bx.loy = fminf(bx.loy, P[i][1]); bx.hiy = fmaxf(bx.hiy, P[i][1]);
    bx.loz = fminf(bx.loz, P[i][2]); bx.hiz = fmaxf(bx.hiz, P[i][2]);
  }
  out = bx;
  // weights of b and c: u = ((x - a) x e2) . n / |n|^2, v = (e1 x (x - a)) . n / |n|^2
  const float e1[3] = {b.x - a.x, b.y - a.y, b.z - a.z}, e2[3] = {c.x - a.x, c.y - a.y, c.z - a.z};
  const float nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2], nz = e1[0] * e2[1] - e1[1] * e2[0];
  const float inv = 1.0f / (nx * nx + ny * ny + nz * nz);
  bary[0] = bary[1] = INFINITY;
  bary[2] = bary[3] = -INFINITY;
  for (int i = 0; i < n; ++i) {
    const float x0 = P[i][0] - a.x, x1 = P[i][1] - a.y, x2 = P[i][2] - a.z;
    const float u = ((x1 * e2[2] - x2 * e2[1]) * nx + (x2 * e2[0] - x0 * e2[2]) * ny + (x0 * e2[1] - x1 * e2[0]) * nz) * inv;
    const float v = ((e1[1] * x2 - e1[2] * x1) * nx + (e1[2] * x0 - e1[0] * x2) * ny + (e1[0] * x1 - e1[1] * x0) * nz) * inv;
    bary[0] = fminf(bary[0], u);
    bary[1] = fminf(bary[1], v);
    bary[2] = fmaxf(bary[2], u);
    bary[3] = fmaxf(bary[3], v);
  }
  return true;
}

// A reference's barycentric range [u0, u1] x [v0, v1] as four 16-bit steps
// of 1/65535, rounded outward by a margin that covers the float32 rounding of
// the clipping and of the weights (1/1024); a sliver (shortest altitude below
// 1e-3 of the coordinates) or a non-finite range gets the whole triangle. The range
// is fixed under any rigid motion of the triangle, so a refit can rebuild
// the reference's box from it.
constexpr uint32_t kBaryWholeLo = 0u, kBaryWholeHi = 0xFFFFFFFFu;

__device__ __forceinline__ uint2 pack_bary(const float4& a, const float4& b, const float4& c, const float r[4]) {
  const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z, e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
  const float e3x = c.x - b.x, e3y = c.y - b.y, e3z = c.z - b.z;
  const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  const float area2 = sqrtf(nx * nx + ny * ny + nz * nz);
  const float lmax = sqrtf(fmaxf(fmaxf(e1x * e1x + e1y * e1y + e1z * e1z, e2x * e2x + e2y * e2y + e2z * e2z),
                                 e3x * e3x + e3y * e3y + e3z * e3z));
  const float cmax = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(b.x))),
                           fmaxf(fmaxf(fabsf(b.y), fabsf(b.z)), fmaxf(fmaxf(fabsf(c.x), fabsf(c.y)), fabsf(c.z))));
  // shortest altitude = |n| / longest edge; at >= 1e-3 of the coordinates the
  // weights' rounding stays well inside the margin
  if (!(area2 > 0.0f) || !(area2 / lmax >= 1e-3f * fmaxf(cmax, 1.0f))) return make_uint2(kBaryWholeLo, kBaryWholeHi);
  const float m = 1.0f / 1024.0f;
  const float u0 = fmaxf(r[0] - m, 0.0f), v0 = fmaxf(r[1] - m, 0.0f), u1 = fminf(r[2] + m, 1.0f),
              v1 = fminf(r[3] + m, 1.0f);
  if (!(u0 <= u1) || !(v0 <= v1)) return make_uint2(kBaryWholeLo, kBaryWholeHi);
  const uint32_t qu0 = (uint32_t)floorf(u0 * 65535.0f), qv0 = (uint32_t)floorf(v0 * 65535.0f);
  const uint32_t qu1 = (uint32_t)ceilf(u1 * 65535.0f), qv1 = (uint32_t)ceilf(v1 * 65535.0f);
  return make_uint2(qu0 | (qv0 << 16), min(qu1, 65535u) | (min(qv1, 65535u) << 16));
}

__device__ __forceinline__ float widen_dn(float x) { return x - 1.9073486328125e-6f * fmaxf(fabsf(x), 1.0f); }
__device__ __forceinline__ float widen_up(float x) { return x + 1.9073486328125e-6f * fmaxf(fabsf(x), 1.0f); }

// One pass per triangle: count (out_box == nullptr) or emit its references.
template <bool kEmit>
__global__ void k_split(const float4* __restrict__ packed, const int32_t* __restrict__ tri_env, int32_t F,
                        const int32_t* __restrict__ bounds, float cells, int max_refs,
                        int32_t* __restrict__ counts,
                        const int32_t* __restrict__ ref_off, int32_t* __restrict__ ref_tri,
                        Box* __restrict__ ref_box, int32_t* __restrict__ ref_env, uint2* __restrict__ ref_bary) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= F) return;
  const int32_t e = tri_env[t];
  const Box tb = tri_box(packed, t);
  float cell = 0.0f;
  if (cells > 0.0f) {
    const int32_t* b = bounds + 6 * (int64_t)e;
    float ext = fmaxf(fmaxf(ord2f(b[3]) - ord2f(b[0]), ord2f(b[4]) - ord2f(b[1])), ord2f(b[5]) - ord2f(b[2]));
    cell = ext / cells;
  }
  const SplitGrid g = split_grid(tb, cell, max_refs);
  int32_t out = kEmit ? ref_off[t] : 0;
  int32_t count = 0;
  if (g.n[0] * g.n[1] * g.n[2] == 1) {
    count = 1;
    if (kEmit) {
      ref_tri[out] = t;
      ref_box[out] = tb;
      ref_env[out] = e;
      ref_bary[out] = make_uint2(kBaryWholeLo, kBaryWholeHi);
    }
  } else {
    const float4 A = packed[3 * (int64_t)t], B = packed[3 * (int64_t)t + 1], C = packed[3 * (int64_t)t + 2];
    for (int i = 0; i < g.n[0]; ++i)
      for (int j = 0; j < g.n[1]; ++j)
        for (int k = 0; k < g.n[2]; ++k) {
          const float lo[3] = {grid_bound(g, 0, i), grid_bound(g, 1, j), grid_bound(g, 2, k)};
          const float hi[3] = {grid_bound(g, 0, i + 1), grid_bound(g, 1, j + 1), grid_bound(g, 2, k + 1)};
          // clip against the cell widened by the same margin, so rounding at
          // the cell faces cannot drop a sliver of the triangle
          const float wlo[3] = {widen_dn(lo[0]), widen_dn(lo[1]), widen_dn(lo[2])};
          const float whi[3] = {widen_up(hi[0]), widen_up(hi[1]), widen_up(hi[2])};
          Box cb;
          float br[4];
          if (!clip_to_cell(A, B, C, wlo, whi, cb, br)) continue;
          if (kEmit) {
            Box r = {fmaxf(widen_dn(cb.lox), tb.lox), fmaxf(widen_dn(cb.loy), tb.loy), fmaxf(widen_dn(cb.loz), tb.loz),
                     fminf(widen_up(cb.hix), tb.hix), fminf(widen_up(cb.hiy), tb.hiy), fminf(widen_up(cb.hiz), tb.hiz)};
            ref_tri[out + count] = t;
            ref_box[out + count] = r;
            ref_env[out + count] = e;
            ref_bary[out + count] = pack_bary(A, B, C, br);
          }
          ++count;
        }
    if (count == 0) {  // cannot happen for a finite triangle; keep it referenced regardless
      count = 1;
      if (kEmit) {
        ref_tri[out] = t;
        ref_box[out] = tb;
        ref_env[out] = e;
        ref_bary[out] = make_uint2(kBaryWholeLo, kBaryWholeHi);
      }
    }
  }
  if (!kEmit) counts[t] = count;
}

// reference offset of each environment's first triangle
__global__ void k_env_ref_off(const int32_t* __restrict__ ref_off, const int32_t* __restrict__ env_tri_off,
                              int32_t E, int32_t F, const int32_t* __restrict__ total, int32_t* __restrict__ out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > E) return;
  int32_t t = env_tri_off[e];
  out[e] = t < F ? ref_off[t] : *total;
}

// ---------------------------------------------------------------- Karras tree
// Inner node li of environment e has global index env_tri_off[e] + li; its
// children are inner nodes (>= 0) or leaves (~sorted position, < 0).
__device__ __forceinline__ int delta(const uint64_t* keys, int64_t base, int32_t n, int32_t a, int32_t b) {
  if (b < 0 || b >= n) return -1;
  uint64_t ka = keys[base + a], kb = keys[base + b];
  if (ka == kb) return 64 + __clz((uint32_t)a ^ (uint32_t)b);
  return __clzll(ka ^ kb);
}

__global__ void k_karras(const uint64_t* __restrict__ keys, int32_t F, int key_shift,
                         const int32_t* __restrict__ env_tri_off, int32_t* __restrict__ left,
                         int32_t* __restrict__ right, int32_t* __restrict__ parent_inner,
                         int32_t* __restrict__ parent_leaf, int32_t* __restrict__ first,
                         int32_t* __restrict__ last) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= F) return;
  int32_t e = (int32_t)(keys[g] >> key_shift);
  int64_t base = env_tri_off[e];
  int32_t n = env_tri_off[e + 1] - (int32_t)base;
  int32_t i = g - (int32_t)base;
  if (i == 0) {
    if (n == 1) parent_leaf[g] = -1;
    else parent_inner[g] = -1;  // root of this environment
  }
  if (i >= n - 1) return;
  int d = (delta(keys, base, n, i, i + 1) - delta(keys, base, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(keys, base, n, i, i - d);
  int32_t lmax = 2;
  while (delta(keys, base, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int32_t l = 0;
  for (int32_t t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, base, n, i, i + (l + t) * d) > dmin) l += t;
  int32_t j = i + l * d;
  int dnode = delta(keys, base, n, i, j);
  int32_t s = 0;
  int32_t t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, base, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int32_t gamma = i + s * d + min(d, 0);
  int32_t lo = min(i, j), hi = max(i, j);
  int32_t lc, rc;
  if (lo == gamma) {
    lc = ~(int32_t)(base + gamma);
    parent_leaf[base + gamma] = g;
  } else {
    lc = (int32_t)(base + gamma);
    parent_inner[base + gamma] = g;
  }
  if (hi == gamma + 1) {
    rc = ~(int32_t)(base + gamma + 1);
    parent_leaf[base + gamma + 1] = g;
  } else {
    rc = (int32_t)(base + gamma + 1);
    parent_inner[base + gamma + 1] = g;
  }
  left[g] = lc;
  right[g] = rc;
  first[g] = (int32_t)base + lo;
  last[g] = (int32_t)base + hi;
}


__device__ __forceinline__ Box load_box_cg(const Box* p) {
  const float* f = reinterpret_cast<const float*>(p);
  Box b;
  b.lox = __ldcg(f);
  b.loy = __ldcg(f + 1);
  b.loz = __ldcg(f + 2);
  b.hix = __ldcg(f + 3);
  b.hiy = __ldcg(f + 4);
  b.hiz = __ldcg(f + 5);
  return b;
}

__device__ __forceinline__ Box box_union(const Box& a, const Box& b) {
  return {fminf(a.lox, b.lox), fminf(a.loy, b.loy), fminf(a.loz, b.loz),
          fmaxf(a.hix, b.hix), fmaxf(a.hiy, b.hiy), fmaxf(a.hiz, b.hiz)};
}

__device__ __forceinline__ void store_box_cg(Box* p, const Box& b) {
  float* f = reinterpret_cast<float*>(p);
  __stcg(f, b.lox);
  __stcg(f + 1, b.loy);
  __stcg(f + 2, b.loz);
  __stcg(f + 3, b.hix);
  __stcg(f + 4, b.hiy);
  __stcg(f + 5, b.hiz);
}

// Bottom-up refit: the second child to arrive at a node computes its box.
__global__ void k_refit(const Box* __restrict__ ref_box, const uint32_t* __restrict__ vals, int32_t F,
                        const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                        const int32_t* __restrict__ parent_inner, const int32_t* __restrict__ parent_leaf,
                        Box* __restrict__ leaf_box, Box* __restrict__ inner_box, int32_t* __restrict__ visits) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  Box b = ref_box[vals[i]];
  store_box_cg(leaf_box + i, b);
  int32_t p = parent_leaf[i];
  int guard = 0;
  while (p >= 0 && guard++ < 4096) {
    __threadfence();
    if (atomicAdd(visits + p, 1) == 0) return;
    __threadfence();
    int32_t l = left[p], r = right[p];
    Box bl = l >= 0 ? load_box_cg(inner_box + l) : load_box_cg(leaf_box + ~l);
    Box br = r >= 0 ? load_box_cg(inner_box + r) : load_box_cg(leaf_box + ~r);
    store_box_cg(inner_box + p, box_union(bl, br));
    p = parent_inner[p];
  }
}

// ---------------------------------------------------------------- collapse
struct QueueItem {
  int32_t ref;  // inner node (>= 0) or ~leaf (single-triangle environment root)
  int32_t env;
};

__device__ __forceinline__ int32_t ref_count(int32_t ref, const int32_t* first, const int32_t* last) {
  return ref >= 0 ? last[ref] - first[ref] + 1 : 1;
}

__device__ __forceinline__ float box_area(const Box& b) {
  float dx = b.hix - b.lox, dy = b.hiy - b.loy, dz = b.hiz - b.loz;
  return dx * dy + dy * dz + dz * dx;
}

constexpr int32_t kSlotEmpty = (int32_t)0x80000000;

// Phase A: open the binary subtree below each queued node into up to 8
// slots, classify them and count. With `choice` (the clustered tree's
// least-cost slots, from build_ploc) the slots follow its decisions;
// otherwise the largest child by surface area is opened until 8 slots.
__global__ void k_collapse_expand(const QueueItem* __restrict__ items, int32_t n_items,
                                  const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                                  const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                                  const Box* __restrict__ inner_box, int leaf_max, int32_t* __restrict__ slots,
                                  int32_t* __restrict__ n_inner, int32_t* __restrict__ n_leaf_tris, int32_t F,
                                  int* __restrict__ err, const uint32_t* __restrict__ choice) {
  int32_t it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  int32_t ref = items[it].ref;
  // every reference must name a node or leaf of this build; anything else is
  // reported instead of being followed
  auto bad = [&](int32_t r) { return r >= 0 ? r >= F : ~r >= F; };
  if (bad(ref)) {
    atomicOr(err, 1);
    slots[8 * (int64_t)it] = kSlotEmpty;
    n_inner[it] = 0;
    n_leaf_tris[it] = 0;
    return;
  }
  int32_t s[8];
  int ns = 0;
  if (ref >= 0) {
    s[0] = left[ref];
    s[1] = right[ref];
    ns = 2;
  } else {
    s[0] = ref;
    ns = 1;
  }
  if (bad(s[0]) || (ns == 2 && bad(s[1]))) {
    atomicOr(err, 1);
    ns = 0;
  }
  if (choice && ns == 2) {
    // follow the least-cost decomposition of the 8 slots: (node, budget) pairs
    int32_t pn[8];
    int pb[8], np = 0;
    const int k8 = (int)((choice[ref] >> 18) & 7u) + 1;
    pn[np] = s[1], pb[np++] = 8 - k8;
    pn[np] = s[0], pb[np++] = k8;
    ns = 0;
    while (np > 0) {
      const int32_t c = pn[--np];
      const int b = pb[np];
      const uint32_t ch = c >= 0 ? choice[c] : 0u;
      if (c < 0 || b <= 1 || ((ch >> (21 + b - 2)) & 1u) || ns + np >= 7) {
        s[ns++] = c;  // one slot (the last guard only bounds a corrupt choice)
        continue;
      }
      if (bad(left[c]) || bad(right[c])) {
        atomicOr(err, 1);
        s[ns++] = c;
        continue;
      }
      const int k = (int)((ch >> (3 * (b - 2))) & 7u) + 1;
      pn[np] = right[c], pb[np++] = b - k;
      pn[np] = left[c], pb[np++] = k;
    }
  }
  while (ns < 8 && !choice) {
    int best = -1;
    float best_area = -1.0f;
    for (int k = 0; k < ns; ++k) {
      int32_t r = s[k];
      if (r >= 0 && ref_count(r, first, last) > leaf_max) {
        float a = box_area(inner_box[r]);
        if (a > best_area) {
          best_area = a;
          best = k;
        }
      }
    }
    if (best < 0) break;
    int32_t r = s[best];
    if (bad(left[r]) || bad(right[r])) {
      atomicOr(err, 1);
      break;
    }
    s[best] = left[r];
    s[ns++] = right[r];
  }
  int ni = 0, nt = 0;
  for (int k = 0; k < 8; ++k) {
    int32_t r = k < ns ? s[k] : kSlotEmpty;
    slots[8 * (int64_t)it + k] = r;
    if (k >= ns) continue;
    int32_t c = ref_count(r, first, last);
    if (r >= 0 && c > leaf_max) ++ni;
    else nt += c;
  }
  n_inner[it] = ni;
  n_leaf_tris[it] = nt;
}

// Phase C: write the wide nodes of this level, the next level's queue and
// the leaf-order triangle permutation.
__global__ void k_collapse_emit(const QueueItem* __restrict__ items, int32_t n_items,
                                const int32_t* __restrict__ slots, const int32_t* __restrict__ inner_off,
                                const int32_t* __restrict__ tri_off, int32_t level_base, int32_t next_base,
                                int32_t tri_base_level, const int32_t* __restrict__ first,
                                const int32_t* __restrict__ last, const Box* __restrict__ inner_box,
                                const Box* __restrict__ leaf_box, int leaf_max, WideNode* __restrict__ nodes,
                                QueueItem* __restrict__ next_items, int32_t* __restrict__ perm,
                                unsigned long long* __restrict__ env_nodes) {
  int32_t it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  QueueItem q = items[it];
  WideNode nd;
  nd.child_base = next_base + inner_off[it];
  nd.tri_base = tri_base_level + tri_off[it];
  uint32_t meta[2] = {0, 0};
  // inner children take slots 0..ni-1 (child k is node child_base + k), then
  // the leaves, then the empty slots
  int ni = 0;
  for (int k = 0; k < 8; ++k) {
    int32_t r = slots[8 * (int64_t)it + k];
    if (r != kSlotEmpty && r >= 0 && ref_count(r, first, last) > leaf_max) ++ni;
  }
  int pos = 0, rank = 0, toff = 0;
  for (int pass = 0; pass < 3; ++pass) {
    for (int k = 0; k < 8; ++k) {
      int32_t r = slots[8 * (int64_t)it + k];
      const bool empty = r == kSlotEmpty;
      const bool inner = !empty && r >= 0 && ref_count(r, first, last) > leaf_max;
      if ((pass == 0) != inner || (pass == 2) != empty) continue;
      uint32_t m;
      Box b;
      if (empty) {
        m = kMetaEmpty;
        b = {kEmptyBoxCoord, kEmptyBoxCoord, kEmptyBoxCoord, kEmptyBoxCoord, kEmptyBoxCoord, kEmptyBoxCoord};
      } else {
        int32_t c = ref_count(r, first, last);
        b = r >= 0 ? inner_box[r] : leaf_box[~r];
        if (inner) {
          m = 0x80u | (uint32_t)ni;
          next_items[inner_off[it] + rank] = {r, q.env};
          ++rank;
        } else {
          int32_t f0 = r >= 0 ? first[r] : ~r;
          m = ((uint32_t)toff << 2) | (uint32_t)(c - 1);
          for (int32_t x = 0; x < c; ++x) perm[nd.tri_base + toff + x] = f0 + x;
          toff += c;
        }
      }
      meta[pos >> 2] |= (m & 0xFFu) << (8 * (pos & 3));
      nd.lox[pos] = b.lox;
      nd.hix[pos] = b.hix;
      nd.loy[pos] = b.loy;
      nd.hiy[pos] = b.hiy;
      nd.loz[pos] = b.loz;
      nd.hiz[pos] = b.hiz;
      ++pos;
    }
  }
  nd.meta_lo = meta[0];
  nd.meta_hi = meta[1];
  nodes[level_base + it] = nd;
  atomicAdd(env_nodes + q.env, 1ull);
}

__global__ void k_gather_tris(const float4* __restrict__ packed, const int32_t* __restrict__ ref_tri,
                              const uint2* __restrict__ ref_bary, const uint32_t* __restrict__ vals,
                              const int32_t* __restrict__ perm, int32_t R, float4* __restrict__ out,
                              int32_t* __restrict__ leaf_tri, uint2* __restrict__ leaf_bary) {
  int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R) return;
  const int32_t ref = vals[perm[k]];
  int64_t t = ref_tri[ref];
  leaf_tri[k] = (int32_t)t;
  if (leaf_bary) leaf_bary[k] = ref_bary[ref];
  out[3 * (int64_t)k] = packed[3 * t];
  out[3 * (int64_t)k + 1] = packed[3 * t + 1];
  out[3 * (int64_t)k + 2] = packed[3 * t + 2];
}

// ---------------------------------------------------------------- compressed nodes
// Child bounds relative to the node's own box: float16 offsets rounded
// outward, or 8-bit steps of a power-of-two scale per axis rounded outward,
// so every stored box contains the exact float32 child box (culling stays
// conservative and ray results stay bit-identical to the float32 nodes).
struct __align__(16) NodeF16 {
  int32_t child_base, tri_base;
  uint32_t meta_lo, meta_hi;
  float ox, oy, oz, pad;
  __half lo_x[8], hi_x[8], lo_y[8], hi_y[8], lo_z[8], hi_z[8];
};
static_assert(sizeof(NodeF16) == 128, "NodeF16 layout");

struct __align__(16) NodeQ8 {
  float ox, oy, oz;
  uint32_t exps;  // biased exponents of the x, y, z scales in bits 0-7, 8-15, 16-23
  int32_t child_base, tri_base;
  uint32_t meta_lo, meta_hi;
  uint8_t lo_x[8], hi_x[8], lo_y[8], hi_y[8], lo_z[8], hi_z[8];
};
static_assert(sizeof(NodeQ8) == 80, "NodeQ8 layout");

__device__ __forceinline__ bool slot_empty(const WideNode& n, int k) {
  return ((((k < 4) ? n.meta_lo : n.meta_hi) >> (8 * (k & 3))) & 0xFFu) == kMetaEmpty;
}

template <int kFmt>
__global__ void k_compress_nodes(const WideNode* __restrict__ in, int64_t n, void* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const WideNode w = in[i];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = 0; k < 8; ++k) {
    if (slot_empty(w, k)) continue;
    lo[0] = fminf(lo[0], w.lox[k]); lo[1] = fminf(lo[1], w.loy[k]); lo[2] = fminf(lo[2], w.loz[k]);
    hi[0] = fmaxf(hi[0], w.hix[k]); hi[1] = fmaxf(hi[1], w.hiy[k]); hi[2] = fmaxf(hi[2], w.hiz[k]);
  }
  for (int a = 0; a < 3; ++a)
    if (!(lo[a] <= hi[a])) lo[a] = hi[a] = 0.0f;  // no valid child (cannot happen)
  if constexpr (kFmt == kNodeFp16) {
    NodeF16 o;
    o.child_base = w.child_base; o.tri_base = w.tri_base; o.meta_lo = w.meta_lo; o.meta_hi = w.meta_hi;
    o.ox = lo[0]; o.oy = lo[1]; o.oz = lo[2]; o.pad = 0.0f;
    const __half inf = __ushort_as_half((unsigned short)0x7C00);
    for (int k = 0; k < 8; ++k) {
      if (slot_empty(w, k)) {
        o.lo_x[k] = o.hi_x[k] = o.lo_y[k] = o.hi_y[k] = o.lo_z[k] = o.hi_z[k] = inf;
        continue;
      }
      o.lo_x[k] = __float2half_rd(__fsub_rd(w.lox[k], lo[0])); o.hi_x[k] = __float2half_ru(__fsub_ru(w.hix[k], lo[0]));
      o.lo_y[k] = __float2half_rd(__fsub_rd(w.loy[k], lo[1])); o.hi_y[k] = __float2half_ru(__fsub_ru(w.hiy[k], lo[1]));
      o.lo_z[k] = __float2half_rd(__fsub_rd(w.loz[k], lo[2])); o.hi_z[k] = __float2half_ru(__fsub_ru(w.hiz[k], lo[2]));
    }
    reinterpret_cast<NodeF16*>(out)[i] = o;
  } else {
    NodeQ8 o;
    o.child_base = w.child_base; o.tri_base = w.tri_base; o.meta_lo = w.meta_lo; o.meta_hi = w.meta_hi;
    o.ox = lo[0]; o.oy = lo[1]; o.oz = lo[2];
    float inv_s[3];
    uint32_t exps = 0;
    for (int a = 0; a < 3; ++a) {
      // scale 2^e with 255 * 2^e >= extent (rounded up)
      const float ext = __fsub_ru(hi[a], lo[a]);
      const float v = __fdiv_ru(ext, 255.0f);
      int e = -126;
      if (v > 0.0f) {
        frexpf(v, &e);
        e = max(-126, min(e, 126));
      }
      exps |= (uint32_t)(e + 127) << (8 * a);
      inv_s[a] = __uint_as_float((uint32_t)(127 - e) << 23);
    }
    o.exps = exps;
    const float* clo[3] = {w.lox, w.loy, w.loz};
    const float* chi[3] = {w.hix, w.hiy, w.hiz};
    uint8_t* qlo[3] = {o.lo_x, o.lo_y, o.lo_z};
    uint8_t* qhi[3] = {o.hi_x, o.hi_y, o.hi_z};
    for (int k = 0; k < 8; ++k)
      for (int a = 0; a < 3; ++a) {
        if (slot_empty(w, k)) {
          qlo[a][k] = 255;
          qhi[a][k] = 0;
          continue;
        }
        const float l = floorf(__fsub_rd(clo[a][k], lo[a]) * inv_s[a]);
        const float h = ceilf(__fsub_ru(chi[a][k], lo[a]) * inv_s[a]);
        qlo[a][k] = (uint8_t)fminf(fmaxf(l, 0.0f), 255.0f);
        qhi[a][k] = (uint8_t)fminf(fmaxf(h, 0.0f), 255.0f);
      }
    reinterpret_cast<NodeQ8*>(out)[i] = o;
  }
}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// device allocations released on scope exit
}  // namespace

ags_status build_scene(ags_context* ctx, ags_scene* sc, const float* base_verts_h, const int32_t* tri_vidx_h,
                       const int32_t* sub_vert_off_h, const float* poses_h, const int32_t* sub_env_h) {
  NvtxRange range("ags build_scene");
  cudaStream_t s = ctx->stream;
  const int32_t E = sc->n_envs;
  const int32_t F = (int32_t)sc->n_tris;
  const int32_t V = (int32_t)sc->n_verts;
  const int32_t J = (int32_t)sc->n_subs;
  DevBufs tmp;

  // persistent buffers (owned by the scene)
  AGS_CHECK(cudaMalloc(&sc->d.world_verts, std::max<int64_t>(V, 1) * sizeof(float4)));
  AGS_CHECK(cudaMalloc(&sc->d.tri_vidx, std::max<int64_t>(3 * (int64_t)F, 1) * sizeof(int32_t)));
  AGS_CHECK(cudaMalloc(&sc->d.env_root, std::max<int32_t>(E, 1) * sizeof(int32_t)));

  float *d_base = nullptr, *d_poses = nullptr, *d_rot = nullptr;
  int32_t *d_sub_vert = nullptr, *d_sub_tri = nullptr, *d_sub_seg = nullptr, *d_sub_env = nullptr,
          *d_env_tri = nullptr;
  AGS_CHECK(tmp.alloc(&d_base, 3 * (size_t)V));
  AGS_CHECK(tmp.alloc(&d_poses, 7 * (size_t)J));
  AGS_CHECK(tmp.alloc(&d_rot, 18 * (size_t)J));
  AGS_CHECK(tmp.alloc(&d_sub_vert, (size_t)J + 1));
  AGS_CHECK(tmp.alloc(&d_sub_tri, (size_t)J + 1));
  AGS_CHECK(tmp.alloc(&d_sub_seg, (size_t)J));
  AGS_CHECK(tmp.alloc(&d_sub_env, (size_t)J));
  AGS_CHECK(tmp.alloc(&d_env_tri, (size_t)E + 1));

  std::vector<int32_t> sub_tri32(J + 1), env_tri32(E + 1);
  for (int32_t j = 0; j <= J; ++j) sub_tri32[j] = (int32_t)sc->sub_tri_off[j];
  for (int32_t e = 0; e <= E; ++e) env_tri32[e] = (int32_t)sc->env_tri_off[e];

  AGS_CHECK(cudaMemcpyAsync(d_base, base_verts_h, 3 * (size_t)V * sizeof(float), cudaMemcpyHostToDevice, s));
  // kept for ags_scene_update_poses: base vertices and sub-mesh vertex offsets on the device
  AGS_CHECK(cudaMalloc(&sc->d.base_verts, std::max<int64_t>(3 * (int64_t)V, 1) * sizeof(float)));
  AGS_CHECK(cudaMalloc(&sc->d.sub_vert_off, ((size_t)J + 1) * sizeof(int32_t)));
  AGS_CHECK(cudaMemcpyAsync(sc->d.base_verts, base_verts_h, 3 * (size_t)V * sizeof(float), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(sc->d.sub_vert_off, sub_vert_off_h, ((size_t)J + 1) * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMalloc(&sc->d.sub_tri_off, ((size_t)J + 1) * sizeof(int32_t)));
  AGS_CHECK(cudaMalloc(&sc->d.sub_poses, std::max<int64_t>(7 * (int64_t)J, 1) * sizeof(float)));
  AGS_CHECK(cudaMemcpyAsync(sc->d.sub_tri_off, sub_tri32.data(), ((size_t)J + 1) * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(sc->d.sub_poses, poses_h, 7 * (size_t)J * sizeof(float), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(d_poses, poses_h, 7 * (size_t)J * sizeof(float), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(d_sub_vert, sub_vert_off_h, ((size_t)J + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(d_sub_tri, sub_tri32.data(), ((size_t)J + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(d_sub_seg, sc->sub_seg.data(), (size_t)J * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(d_sub_env, sub_env_h, (size_t)J * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(d_env_tri, env_tri32.data(), ((size_t)E + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(sc->d.tri_vidx, tri_vidx_h, 3 * (size_t)F * sizeof(int32_t), cudaMemcpyHostToDevice, s));

  // a1: transform
  if (J > 0) k_submesh_rotations<<<blocks_for(J, 128), 128, 0, s>>>(d_poses, J, d_rot);
  if (V > 0)
    k_transform_vertices<<<blocks_for(V, 256), 256, 0, s>>>(d_base, V, d_sub_vert, J, d_rot, d_poses,
                                                            sc->d.world_verts);
  AGS_CHECK(cudaGetLastError());

  sc->env_nodes.assign(E, 0);
  sc->env_ref_off.assign(E + 1, 0);
  if (F == 0) {
    std::vector<int32_t> env_root(E, -1);
    AGS_CHECK(cudaMemcpyAsync(sc->d.env_root, env_root.data(), (size_t)std::max(E, 1) * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s));
    sc->node_format = (int)(sc->flags & 0xFFu);
    AGS_CHECK(cudaMalloc(&sc->d.nodes, sizeof(WideNode)));
    sc->n_nodes = 0;
    sc->n_refs = 0;
    AGS_CHECK(cudaStreamSynchronize(s));
    return AGS_OK;
  }

  // packed triangles in input order
  float4* d_packed = nullptr;
  int32_t* d_tri_env = nullptr;
  AGS_CHECK(tmp.alloc(&d_packed, 3 * (size_t)F));
  AGS_CHECK(tmp.alloc(&d_tri_env, (size_t)F));
  k_pack_triangles<<<blocks_for(F, 256), 256, 0, s>>>(sc->d.tri_vidx, F, sc->d.world_verts, d_sub_tri, J, d_sub_seg,
                                                      d_sub_env, d_env_tri, d_packed, d_tri_env);

  // per-environment bounds of triangle boxes' centres: split cell size and Morton frame
  Box* d_tbox = nullptr;
  int32_t* d_bounds = nullptr;
  AGS_CHECK(tmp.alloc(&d_tbox, (size_t)F));
  AGS_CHECK(tmp.alloc(&d_bounds, 6 * (size_t)E));
  k_tri_boxes<<<blocks_for(F, 256), 256, 0, s>>>(d_packed, F, d_tbox);
  k_init_bounds<<<blocks_for(E, 128), 128, 0, s>>>(d_bounds, E);
  k_env_bounds<<<blocks_for(F, 256), 256, 0, s>>>(d_tbox, d_tri_env, F, d_bounds);

  // references: large triangles split into clipped cells
  const uint32_t split_code = (sc->flags >> 12) & 0xFFu;
  const float cells = split_code == 1 ? 0.0f : (split_code == 0 ? (float)kDefaultSplitCells : (float)split_code);
  int32_t *d_ref_count = nullptr, *d_ref_tot = nullptr, *d_env_ref = nullptr;
  AGS_CHECK(tmp.alloc(&d_ref_count, (size_t)F));
  AGS_CHECK(tmp.alloc(&d_ref_tot, 1));
  AGS_CHECK(tmp.alloc(&d_env_ref, (size_t)E + 1));
  void* d_scan_f = nullptr;
  AGS_CHECK(tmp.alloc(reinterpret_cast<char**>(&d_scan_f), scan_temp_bytes(F)));
  // references per triangle are capped so that their total stays below 2^31
  const int max_refs = (int)std::max<int64_t>(1, std::min<int64_t>(kSplitMaxRefs, ((1ll << 31) - 2 - F) / F + 1));
  k_split<false><<<blocks_for(F, 128), 128, 0, s>>>(d_packed, d_tri_env, F, d_bounds, cells, max_refs, d_ref_count,
                                                   nullptr, nullptr, nullptr, nullptr, nullptr);
  AGS_CHECK(cudaGetLastError());
  AGS_CHECK(exclusive_scan(d_ref_count, F, d_ref_tot, d_scan_f, s));
  k_env_ref_off<<<blocks_for((int64_t)E + 1, 128), 128, 0, s>>>(d_ref_count, d_env_tri, E, F, d_ref_tot, d_env_ref);
  std::vector<int32_t> env_ref32(E + 1);
  AGS_CHECK(cudaMemcpyAsync(env_ref32.data(), d_env_ref, ((size_t)E + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  AGS_CHECK(cudaStreamSynchronize(s));
  const int32_t R = env_ref32[E];
  if (R < F) {
    set_error("reference splitting produced too few references");
    return AGS_ERR_CUDA;
  }
  for (int32_t e = 0; e <= E; ++e) sc->env_ref_off[e] = env_ref32[e];
  sc->n_refs = R;
  int32_t *d_ref_tri = nullptr, *d_ref_env = nullptr;
  Box* d_ref_box = nullptr;
  uint2* d_ref_bary = nullptr;
  AGS_CHECK(tmp.alloc(&d_ref_tri, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_ref_env, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_ref_box, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_ref_bary, (size_t)R));
  k_split<true><<<blocks_for(F, 128), 128, 0, s>>>(d_packed, d_tri_env, F, d_bounds, cells, max_refs, nullptr,
                                                  d_ref_count, d_ref_tri, d_ref_box, d_ref_env, d_ref_bary);
  AGS_CHECK(cudaGetLastError());

  // roots and level-0 queue (environments with at least one reference)
  std::vector<int32_t> env_root(E, -1);
  std::vector<QueueItem> q0;
  int64_t max_env_refs = 0;
  for (int32_t e = 0; e < E; ++e) {
    int64_t n = sc->env_ref_off[e + 1] - sc->env_ref_off[e];
    max_env_refs = std::max(max_env_refs, n);
    if (n <= 0) continue;
    env_root[e] = (int32_t)q0.size();
    int32_t base = (int32_t)sc->env_ref_off[e];
    q0.push_back({n >= 2 ? base : ~base, e});
  }
  AGS_CHECK(cudaMemcpyAsync(sc->d.env_root, env_root.data(), (size_t)std::max(E, 1) * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));

  // a2: Morton codes of reference centres over each environment's bounds
  int env_bits = 0;
  while ((1ll << env_bits) < E) ++env_bits;
  int bits = 10;
  if (max_env_refs > (1ll << 20)) bits = std::min(21, (64 - env_bits) / 3);
  bits = std::min(bits, (64 - env_bits) / 3);
  int key_shift = 3 * bits;
  int end_bit = key_shift + env_bits;
  k_init_bounds<<<blocks_for(E, 128), 128, 0, s>>>(d_bounds, E);
  k_env_bounds<<<blocks_for(R, 256), 256, 0, s>>>(d_ref_box, d_ref_env, R, d_bounds);
  uint64_t *d_keys = nullptr, *d_keys2 = nullptr;
  uint32_t *d_vals = nullptr, *d_vals2 = nullptr;
  AGS_CHECK(tmp.alloc(&d_keys, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_keys2, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_vals, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_vals2, (size_t)R));
  k_morton<<<blocks_for(R, 256), 256, 0, s>>>(d_ref_box, d_ref_env, R, d_bounds, bits, d_keys, d_vals);
  AGS_CHECK(cudaGetLastError());
  void* d_sort_tmp = nullptr;
  AGS_CHECK(tmp.alloc(reinterpret_cast<char**>(&d_sort_tmp), sort_temp_bytes(R)));
  AGS_CHECK(sort_pairs(d_keys, d_vals, d_keys2, d_vals2, R, end_bit, d_sort_tmp, s));

  // binary radix tree per environment (over its references)
  int32_t *d_left, *d_right, *d_pin, *d_pleaf, *d_first, *d_last, *d_visits;
  AGS_CHECK(tmp.alloc(&d_left, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_right, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_pin, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_pleaf, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_first, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_last, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_visits, (size_t)R));
  AGS_CHECK(cudaMemsetAsync(d_visits, 0, (size_t)R * sizeof(int32_t), s));
  Box *d_leaf_box, *d_inner_box;
  AGS_CHECK(tmp.alloc(&d_leaf_box, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_inner_box, (size_t)R));
  const int leaf_max = ((sc->flags >> 8) & 0xFu) ? (int)((sc->flags >> 8) & 0xFu) : kDefaultLeafTris;
  uint32_t* d_choice = nullptr;  // least-cost wide-node slots (clustered tree only)
  if (sc->flags & AGS_BUILD_LBVH) {
    // Morton radix tree (Karras 2012) and an atomic bottom-up refit
    k_karras<<<blocks_for(R, 256), 256, 0, s>>>(d_keys, R, key_shift, d_env_ref, d_left, d_right, d_pin, d_pleaf,
                                                d_first, d_last);
    k_refit<<<blocks_for(R, 256), 256, 0, s>>>(d_ref_box, d_vals, R, d_left, d_right, d_pin, d_pleaf, d_leaf_box,
                                               d_inner_box, d_visits);
    AGS_CHECK(cudaGetLastError());
  } else {
    // locally-ordered clustering (default): lower surface-area cost
    std::vector<int32_t> roots;
    if (!(sc->flags & AGS_BUILD_GREEDY_COLLAPSE)) AGS_CHECK(tmp.alloc(&d_choice, (size_t)R));
    ags_status st = build_ploc(d_keys, d_vals, R, key_shift, d_env_ref, E, d_ref_box, d_leaf_box, d_left, d_right,
                               d_first, d_last, d_inner_box, roots, s, d_choice, leaf_max,
                               16 << ((sc->flags >> 23) & 3u));
    if (st != AGS_OK) return st;
    for (QueueItem& q : q0) {
      if (q.ref < 0) continue;  // a single reference: the leaf keeps its position
      if (roots[q.env] < 0 || roots[q.env] >= R) {
        set_error("clustering left an environment without a root");
        return AGS_ERR_CUDA;
      }
      q.ref = roots[q.env];
    }
  }

  // collapse into 8-wide nodes, level by level
  // wide nodes: at most R/(L+1) + E without inner children (each covers more
  // than L references, or is a root), and every node with inner children has
  // 8 slots, which bounds those by (R + R/(L+1) + E)/7
  const double leafonly = (double)R / (leaf_max + 1) + E;
  int64_t node_cap = (int64_t)(leafonly + ((double)R + leafonly) / 7.0) + 2 * (int64_t)E + 64;
  WideNode* d_nodes_tmp = nullptr;
  AGS_CHECK(tmp.alloc(&d_nodes_tmp, (size_t)node_cap));
  QueueItem *d_q = nullptr, *d_q2 = nullptr;
  int64_t q_cap = node_cap;
  AGS_CHECK(tmp.alloc(&d_q, (size_t)q_cap));
  AGS_CHECK(tmp.alloc(&d_q2, (size_t)q_cap));
  int32_t *d_slots, *d_ninner, *d_ntris, *d_perm, *d_tot;
  int* d_err = nullptr;
  AGS_CHECK(tmp.alloc(&d_err, 1));
  AGS_CHECK(tmp.alloc(&d_slots, 8 * (size_t)q_cap));
  AGS_CHECK(tmp.alloc(&d_ninner, (size_t)q_cap));
  AGS_CHECK(tmp.alloc(&d_ntris, (size_t)q_cap));
  AGS_CHECK(tmp.alloc(&d_perm, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_tot, 2));
  void* d_scan_tmp = nullptr;
  AGS_CHECK(tmp.alloc(reinterpret_cast<char**>(&d_scan_tmp), scan_temp_bytes(q_cap)));
  unsigned long long* d_env_nodes = nullptr;
  AGS_CHECK(tmp.alloc(&d_env_nodes, (size_t)E));

  // the least-cost slots may leave nodes with fewer than 8 slots; should they
  // outgrow the bound above, the collapse is redone greedily
  int32_t level_base = 0, tri_level_base = 0;
  for (bool again = true; again;) {
  again = false;
  AGS_CHECK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  AGS_CHECK(cudaMemsetAsync(d_env_nodes, 0, (size_t)E * sizeof(unsigned long long), s));
  AGS_CHECK(cudaMemcpyAsync(d_q, q0.data(), q0.size() * sizeof(QueueItem), cudaMemcpyHostToDevice, s));
  int32_t n_items = (int32_t)q0.size();
  level_base = 0;
  tri_level_base = 0;
  int levels = 0;
  sc->level_off.assign(1, 0);
  while (n_items > 0) {
    if (++levels > 4096) {
      set_error("BVH collapse did not terminate");
      return AGS_ERR_CUDA;
    }
    k_collapse_expand<<<blocks_for(n_items, 128), 128, 0, s>>>(d_q, n_items, d_left, d_right, d_first, d_last,
                                                              d_inner_box, leaf_max, d_slots, d_ninner, d_ntris,
                                                              R, d_err, d_choice);
    AGS_CHECK(cudaGetLastError());
    AGS_CHECK(exclusive_scan(d_ninner, n_items, d_tot, d_scan_tmp, s));
    AGS_CHECK(exclusive_scan(d_ntris, n_items, d_tot + 1, d_scan_tmp, s));
    int32_t tot[3];
    AGS_CHECK(cudaMemcpyAsync(tot, d_tot, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AGS_CHECK(cudaMemcpyAsync(tot + 2, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AGS_CHECK(cudaStreamSynchronize(s));
    if (tot[2] != 0) {
      set_error("BVH collapse met an out-of-range node reference");
      return AGS_ERR_CUDA;
    }
    if (tot[0] < 0 || tot[1] < 0 || (int64_t)tri_level_base + tot[1] > R) {
      set_error("BVH collapse produced inconsistent counts");
      return AGS_ERR_CUDA;
    }
    int32_t next_base = level_base + n_items;
    if ((int64_t)next_base + tot[0] > node_cap) {
      if (d_choice) {
        d_choice = nullptr;
        again = true;
        break;
      }
      set_error("BVH node capacity exceeded");
      return AGS_ERR_CUDA;
    }
    k_collapse_emit<<<blocks_for(n_items, 128), 128, 0, s>>>(
        d_q, n_items, d_slots, d_ninner, d_ntris, level_base, next_base, tri_level_base, d_first, d_last,
        d_inner_box, d_leaf_box, leaf_max, d_nodes_tmp, d_q2, d_perm, d_env_nodes);
    AGS_CHECK(cudaGetLastError());
    std::swap(d_q, d_q2);
    level_base = next_base;
    sc->level_off.push_back(level_base);
    tri_level_base += tot[1];
    n_items = tot[0];
  }
  }
  if (tri_level_base != R) {
    set_error("BVH collapse lost references");
    return AGS_ERR_CUDA;
  }
  sc->n_nodes = level_base;
  sc->node_format = (int)(sc->flags & 0xFFu);
  AGS_CHECK(cudaMalloc(&sc->d.nodes, std::max<int64_t>(sc->n_nodes, 1) * node_bytes_of(sc->node_format)));
  if (sc->node_format == kNodeFp32) {
    AGS_CHECK(cudaMemcpyAsync(sc->d.nodes, d_nodes_tmp, (size_t)sc->n_nodes * sizeof(WideNode),
                              cudaMemcpyDeviceToDevice, s));
  } else if (sc->n_nodes > 0) {
    if (sc->node_format == kNodeFp16)
      k_compress_nodes<kNodeFp16><<<blocks_for(sc->n_nodes, 128), 128, 0, s>>>(d_nodes_tmp, sc->n_nodes, sc->d.nodes);
    else
      k_compress_nodes<kNodeQ8><<<blocks_for(sc->n_nodes, 128), 128, 0, s>>>(d_nodes_tmp, sc->n_nodes, sc->d.nodes);
    AGS_CHECK(cudaGetLastError());
  }
  AGS_CHECK(cudaMalloc(&sc->d.tris, std::max<int64_t>(3 * (int64_t)R, 1) * sizeof(float4)));
  AGS_CHECK(cudaMalloc(&sc->d.leaf_tri, std::max<int64_t>(R, 1) * sizeof(int32_t)));
  if (sc->node_format == kNodeFp32)  // refit (float32 nodes only) rebuilds split boxes from these
    AGS_CHECK(cudaMalloc(&sc->d.leaf_bary, std::max<int64_t>(R, 1) * sizeof(uint2)));
  k_gather_tris<<<blocks_for(R, 256), 256, 0, s>>>(d_packed, d_ref_tri, d_ref_bary, d_vals, d_perm, R, sc->d.tris,
                                                   sc->d.leaf_tri, sc->d.leaf_bary);
  AGS_CHECK(cudaGetLastError());
  std::vector<unsigned long long> env_nodes(E);
  AGS_CHECK(cudaMemcpyAsync(env_nodes.data(), d_env_nodes, (size_t)E * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s));
  AGS_CHECK(cudaStreamSynchronize(s));
  for (int32_t e = 0; e < E; ++e) sc->env_nodes[e] = (int64_t)env_nodes[e];
  if (sc->node_format == kNodeFp32) return tree_cost(ctx, sc, &sc->tree_cost_built);
  return AGS_OK;
}

namespace {

// new world xyz of every leaf-order triangle copy (the w words keep segment and index)
__global__ void k_repack_tris(const int32_t* __restrict__ leaf_tri, const int32_t* __restrict__ vidx, int32_t R,
                              const float4* __restrict__ world, float4* __restrict__ tris) {
  int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R) return;
  const int64_t t = leaf_tri[k];
  for (int c = 0; c < 3; ++c) {
    const float4 v = world[vidx[3 * t + c]];
    float4 o = tris[3 * (int64_t)k + c];
    o.x = v.x;
    o.y = v.y;
    o.z = v.z;
    tris[3 * (int64_t)k + c] = o;
  }
}

// Box of one leaf reference at the triangle's current position: the corners
// of its barycentric range a + u e1 + v e2 (widened by the float32 rounding
// of that sum), cut back to the triangle's own box. The range holds the
// reference's piece of the triangle, and the pieces of a triangle's
// references cover it, so culling stays conservative after any motion.
__device__ Box ref_box_at(const float4* __restrict__ tris, int32_t k, uint2 q) {
  const Box tb = tri_box(tris, k);
  if (q.x == kBaryWholeLo && q.y == kBaryWholeHi) return tb;
  const float4 a = tris[3 * (int64_t)k], b = tris[3 * (int64_t)k + 1], c = tris[3 * (int64_t)k + 2];
  const float us[2] = {(float)(q.x & 0xFFFFu) / 65535.0f, (float)(q.y & 0xFFFFu) / 65535.0f};
  const float vs[2] = {(float)(q.x >> 16) / 65535.0f, (float)(q.y >> 16) / 65535.0f};
  Box r = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const float x = a.x + us[i] * (b.x - a.x) + vs[j] * (c.x - a.x);
      const float y = a.y + us[i] * (b.y - a.y) + vs[j] * (c.y - a.y);
      const float z = a.z + us[i] * (b.z - a.z) + vs[j] * (c.z - a.z);
      r.lox = fminf(r.lox, x); r.loy = fminf(r.loy, y); r.loz = fminf(r.loz, z);
      r.hix = fmaxf(r.hix, x); r.hiy = fmaxf(r.hiy, y); r.hiz = fmaxf(r.hiz, z);
    }
  r.lox = fmaxf(widen_dn(r.lox), tb.lox); r.loy = fmaxf(widen_dn(r.loy), tb.loy); r.loz = fmaxf(widen_dn(r.loz), tb.loz);
  r.hix = fminf(widen_up(r.hix), tb.hix); r.hiy = fminf(widen_up(r.hiy), tb.hiy); r.hiz = fminf(widen_up(r.hiz), tb.hiz);
  return r;
}

// Rigid motion of each sub-mesh from its build pose to the new one: x -> R_rel (x - p_old) + p_new with R_rel =
// R(q_new) R(q_old)^T, stored as 16 floats: R_rel row-major, p_old, p_new,
// and 1 when the pose is bit-for-bit unchanged (the vertices do not move).
__device__ __forceinline__ void quat_matrix(const float* q, float R[9]) {
  const float x = q[0], y = q[1], z = q[2], w = q[3];
  const float s = 2.0f / (x * x + y * y + z * z + w * w);
  R[0] = 1.0f - s * (y * y + z * z); R[1] = s * (x * y - z * w);        R[2] = s * (x * z + y * w);
  R[3] = s * (x * y + z * w);        R[4] = 1.0f - s * (x * x + z * z); R[5] = s * (y * z - x * w);
  R[6] = s * (x * z - y * w);        R[7] = s * (y * z + x * w);        R[8] = 1.0f - s * (x * x + y * y);
}

__global__ void k_relative_motion(const float* __restrict__ old_poses, const float* __restrict__ new_poses, int32_t J,
                                  float* __restrict__ motion) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  const float* po = old_poses + 7 * (int64_t)j;
  const float* pn = new_poses + 7 * (int64_t)j;
  float* m = motion + 16 * (int64_t)j;
  bool same = true;
  for (int k = 0; k < 7; ++k) same &= __float_as_uint(po[k]) == __float_as_uint(pn[k]);
  float Ro[9], Rn[9];
  quat_matrix(po + 3, Ro);
  quat_matrix(pn + 3, Rn);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) m[3 * r + c] = Rn[3 * r] * Ro[3 * c] + Rn[3 * r + 1] * Ro[3 * c + 1] + Rn[3 * r + 2] * Ro[3 * c + 2];
  m[9] = po[0]; m[10] = po[1]; m[11] = po[2];
  m[12] = pn[0]; m[13] = pn[1]; m[14] = pn[2];
  m[15] = same ? 1.0f : 0.0f;
}

// The box b moved by a sub-mesh's motion: the box around its eight moved
// corners, widened by 256 u (|corner| + |p_old| + |p_new|) per axis, which
// bounds the float32 rounding of R_rel against the exact relative rotation
// and of the world vertices at both poses.
__device__ Box moved_box(const Box& b, const float* __restrict__ m) {
  Box r = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  const float pm = fmaxf(fmaxf(fabsf(m[9]), fabsf(m[10])), fabsf(m[11])) +
                   fmaxf(fmaxf(fabsf(m[12]), fabsf(m[13])), fabsf(m[14]));
  float cm = 0.0f;
  for (int i = 0; i < 8; ++i) {
    const float cx = (i & 1) ? b.hix : b.lox, cy = (i & 2) ? b.hiy : b.loy, cz = (i & 4) ? b.hiz : b.loz;
    cm = fmaxf(cm, fmaxf(fmaxf(fabsf(cx), fabsf(cy)), fabsf(cz)));
    const float dx = cx - m[9], dy = cy - m[10], dz = cz - m[11];
    const float x = m[0] * dx + m[1] * dy + m[2] * dz + m[12];
    const float y = m[3] * dx + m[4] * dy + m[5] * dz + m[13];
    const float z = m[6] * dx + m[7] * dy + m[8] * dz + m[14];
    r.lox = fminf(r.lox, x); r.loy = fminf(r.loy, y); r.loz = fminf(r.loz, z);
    r.hix = fmaxf(r.hix, x); r.hiy = fmaxf(r.hiy, y); r.hiz = fmaxf(r.hiz, z);
  }
  const float w = 256.0f * 5.96046448e-8f * (cm + pm);
  r.lox -= w; r.loy -= w; r.loz -= w;
  r.hix += w; r.hiy += w; r.hiz += w;
  return r;
}

// Refit one level of float32 wide nodes: each slot's box becomes the union of
// its child node's slots (already refitted: levels run from the deepest up)
// or, for a leaf slot, of its references' boxes. A reference's piece of its
// triangle lies in its barycentric-range box and in the slot's box as built,
// moved with the reference's sub-mesh from its build pose, so it lies in
// their intersection; a sub-mesh back at its build pose keeps the built box.
// Moving from the build pose (not from the last refit) keeps the rotation's
// widening of the boxes from adding up over many updates.
__global__ void k_refit_level(WideNode* __restrict__ nodes, const WideNode* __restrict__ built, int32_t begin,
                              int32_t end, const float4* __restrict__ tris,
                              const uint2* __restrict__ leaf_bary, const int32_t* __restrict__ leaf_tri,
                              const int32_t* __restrict__ sub_tri_off, int32_t J, const float* __restrict__ motion,
                              int32_t n_nodes, int32_t n_tris, int* __restrict__ err) {
  const int32_t i = begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= end) return;
  WideNode& n = nodes[i];
  const uint32_t b0 = n.meta_lo & 0xFFu;
  const int ni = (b0 & 0x80u) ? (int)min(b0 & 0xFu, 8u) : 0;
  for (int k = 0; k < 8; ++k) {
    const uint32_t m = (((k < 4) ? n.meta_lo : n.meta_hi) >> (8 * (k & 3))) & 0xFFu;
    if (m == kMetaEmpty) continue;
    Box b = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    if (k < ni) {
      const int32_t c = n.child_base + k;
      if (c < 0 || c >= n_nodes) {
        atomicOr(err, 1);
        continue;
      }
      const WideNode& ch = nodes[c];
      for (int q = 0; q < 8; ++q) {
        const uint32_t mq = (((q < 4) ? ch.meta_lo : ch.meta_hi) >> (8 * (q & 3))) & 0xFFu;
        if (mq == kMetaEmpty) continue;
        b.lox = fminf(b.lox, ch.lox[q]); b.loy = fminf(b.loy, ch.loy[q]); b.loz = fminf(b.loz, ch.loz[q]);
        b.hix = fmaxf(b.hix, ch.hix[q]); b.hiy = fmaxf(b.hiy, ch.hiy[q]); b.hiz = fmaxf(b.hiz, ch.hiz[q]);
      }
    } else {
      const int32_t start = n.tri_base + (int32_t)(m >> 2), cnt = (int32_t)(m & 3u) + 1;
      if (start < 0 || start + cnt > n_tris) {
        atomicOr(err, 1);
        continue;
      }
      const WideNode& nb = built[i];
      const Box prev = {nb.lox[k], nb.loy[k], nb.loz[k], nb.hix[k], nb.hiy[k], nb.hiz[k]};
      for (int32_t x = 0; x < cnt; ++x) {
        Box tb = ref_box_at(tris, start + x, leaf_bary[start + x]);
        const int32_t j = upper_bound_i32(sub_tri_off + 1, J, leaf_tri[start + x]);
        if (j < J) {
          const float* m = motion + 16 * (int64_t)j;
          const Box mb = m[15] != 0.0f ? prev : moved_box(prev, m);
          const Box ib = {fmaxf(tb.lox, mb.lox), fmaxf(tb.loy, mb.loy), fmaxf(tb.loz, mb.loz),
                          fminf(tb.hix, mb.hix), fminf(tb.hiy, mb.hiy), fminf(tb.hiz, mb.hiz)};
          if (ib.lox <= ib.hix && ib.loy <= ib.hiy && ib.loz <= ib.hiz) tb = ib;
        }
        b.lox = fminf(b.lox, tb.lox); b.loy = fminf(b.loy, tb.loy); b.loz = fminf(b.loz, tb.loz);
        b.hix = fmaxf(b.hix, tb.hix); b.hiy = fmaxf(b.hiy, tb.hiy); b.hiz = fmaxf(b.hiz, tb.hiz);
      }
    }
    n.lox[k] = b.lox; n.loy[k] = b.loy; n.loz[k] = b.loz;
    n.hix[k] = b.hix; n.hiy[k] = b.hiy; n.hiz[k] = b.hiz;
  }
}

}  // namespace

ags_status transform_vertices(const float* base_dev, int32_t V, const int32_t* sub_vert_off_dev, int32_t J,
                              const float* poses_dev, float4* world_dev, cudaStream_t s) {
  DevBufs tmp;
  float* d_rot = nullptr;
  AGS_CHECK(tmp.alloc(&d_rot, 18 * (size_t)std::max(J, 1)));
  if (J > 0) k_submesh_rotations<<<blocks_for(J, 128), 128, 0, s>>>(poses_dev, J, d_rot);
  if (V > 0)
    k_transform_vertices<<<blocks_for(V, 256), 256, 0, s>>>(base_dev, V, sub_vert_off_dev, J, d_rot, poses_dev,
                                                            world_dev);
  AGS_CHECK(cudaGetLastError());
  AGS_CHECK(cudaStreamSynchronize(s));  // the scratch is freed on return
  return AGS_OK;
}

namespace {
// Per node: the collapse's cost of its child boxes (inner: node weight x area; leaf: triangle weight x
// count x area; area as in the collapse, dx dy + dy dz + dz dx), summed in double.
__global__ void k_tree_cost(const WideNode* __restrict__ nodes, int32_t n, double* __restrict__ out) {
  double c = 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const WideNode& nd = nodes[i];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t m = ((k < 4 ? nd.meta_lo : nd.meta_hi) >> (8 * (k & 3))) & 0xFFu;
      if (m == kMetaEmpty) continue;
      const double dx = (double)nd.hix[k] - nd.lox[k], dy = (double)nd.hiy[k] - nd.loy[k],
                   dz = (double)nd.hiz[k] - nd.loz[k];
      const double area = dx * dy + dy * dz + dz * dx;
      c += (m & 0x80u) ? (double)kSahNodeCost * area : (double)kSahTriCost * (double)((m & 3u) + 1) * area;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c != 0.0) atomicAdd(out, c);
}
}  // namespace

ags_status tree_cost(ags_context* ctx, const ags_scene* sc, double* cost) {
  *cost = 0.0;
  if (sc->node_format != kNodeFp32 || sc->n_nodes <= 0) return AGS_OK;
  cudaStream_t s = ctx->stream;
  DevBufs tmp;
  double* d_cost = nullptr;
  AGS_CHECK(tmp.alloc(&d_cost, 1));
  AGS_CHECK(cudaMemsetAsync(d_cost, 0, sizeof(double), s));
  const int blocks = (int)std::min<int64_t>(blocks_for(sc->n_nodes, 256), 4096);
  k_tree_cost<<<blocks, 256, 0, s>>>(static_cast<const WideNode*>(sc->d.nodes), (int32_t)sc->n_nodes, d_cost);
  AGS_CHECK(cudaGetLastError());
  AGS_CHECK(cudaMemcpyAsync(cost, d_cost, sizeof(double), cudaMemcpyDeviceToHost, s));
  AGS_CHECK(cudaStreamSynchronize(s));
  return AGS_OK;
}

ags_status refit_scene(ags_context* ctx, ags_scene* sc, const float* poses_h) {
  NvtxRange range("ags refit_scene");
  cudaStream_t s = ctx->stream;
  if (!sc->d.nodes_build && sc->n_nodes > 0) {
    AGS_CHECK(cudaMalloc(&sc->d.nodes_build, (size_t)sc->n_nodes * sizeof(WideNode)));
    AGS_CHECK(cudaMemcpyAsync(sc->d.nodes_build, sc->d.nodes, (size_t)sc->n_nodes * sizeof(WideNode),
                              cudaMemcpyDeviceToDevice, s));
  }
  const int32_t V = (int32_t)sc->n_verts, J = (int32_t)sc->n_subs, R = (int32_t)sc->n_refs;
  DevBufs tmp;
  float *d_poses = nullptr, *d_rot = nullptr, *d_motion = nullptr;
  int* d_err = nullptr;
  AGS_CHECK(tmp.alloc(&d_poses, 7 * (size_t)std::max(J, 1)));
  AGS_CHECK(tmp.alloc(&d_rot, 18 * (size_t)std::max(J, 1)));
  AGS_CHECK(tmp.alloc(&d_motion, 16 * (size_t)std::max(J, 1)));
  AGS_CHECK(tmp.alloc(&d_err, 1));
  AGS_CHECK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  if (J > 0) AGS_CHECK(cudaMemcpyAsync(d_poses, poses_h, 7 * (size_t)J * sizeof(float), cudaMemcpyHostToDevice, s));
  if (J > 0) k_submesh_rotations<<<blocks_for(J, 128), 128, 0, s>>>(d_poses, J, d_rot);
  if (J > 0) k_relative_motion<<<blocks_for(J, 128), 128, 0, s>>>(sc->d.sub_poses, d_poses, J, d_motion);
  if (V > 0)
    k_transform_vertices<<<blocks_for(V, 256), 256, 0, s>>>(sc->d.base_verts, V, sc->d.sub_vert_off, J, d_rot, d_poses,
                                                            sc->d.world_verts);
  if (R > 0) k_repack_tris<<<blocks_for(R, 256), 256, 0, s>>>(sc->d.leaf_tri, sc->d.tri_vidx, R, sc->d.world_verts,
                                                              sc->d.tris);
  for (size_t l = sc->level_off.size(); l-- > 1;) {
    const int32_t b = (int32_t)sc->level_off[l - 1], e = (int32_t)sc->level_off[l];
    if (e > b)
      k_refit_level<<<blocks_for(e - b, 128), 128, 0, s>>>(static_cast<WideNode*>(sc->d.nodes), sc->d.nodes_build, b,
                                                           e, sc->d.tris,
                                                           sc->d.leaf_bary, sc->d.leaf_tri, sc->d.sub_tri_off, J,
                                                           d_motion, (int32_t)sc->n_nodes, R, d_err);
  }

  AGS_CHECK(cudaGetLastError());
  int err = 0;
  AGS_CHECK(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  AGS_CHECK(cudaStreamSynchronize(s));
  if (err) {
    set_error("refit met an out-of-range node or triangle index");
    return AGS_ERR_CUDA;
  }
  return AGS_OK;
}

}  // namespace ags

// ---------------------------------------------------------------- allocation-free transform
// ags_transform_vertices_noalloc runs the same two transform kernels as the
// scene build, but keeps their per-sub-mesh scratch (the float-float rotation
// of each pose, 18 floats) in this file-scope device array instead of memory
// from cudaMalloc. Every GPU that loads the library holds the array until the
// process exits: 18 floats x 65536 sub-meshes = 4.5 MiB.
#include <mutex>

namespace {
constexpr int32_t kNoAllocMaxSubmeshes = 65536;
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

static __device__ __align__(256) float ags_noalloc_rot_scratch[18 * kNoAllocMaxSubmeshes];

namespace ags {
namespace {

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `device`, looked up once per device
// with that device current (host code cannot use the symbol itself: on the
// host it names a stand-in, not device memory).
ags_status noalloc_scratch(int device, float** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) {
    set_error("ags_transform_vertices_noalloc: device index beyond the supported 64");
    return AGS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    // the address is only valid on the device current at the lookup: never
    // cache one taken with another device current
    int cur = -1;
    cudaError_t ce = cudaGetDevice(&cur);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    if (cur != device) {
      set_error("ags_transform_vertices_noalloc: the context's device is not current");
      return AGS_ERR_CUDA;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, ags_noalloc_rot_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(ags_noalloc_rot_scratch)");
    g_noalloc_ptr[device] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[device];
  return AGS_OK;
}

}  // namespace
}  // namespace ags

extern "C" ags_status ags_transform_vertices_noalloc(ags_context* ctx, const float* base_vertices_dev,
                                                     int32_t n_vertices, const int32_t* submesh_vertex_offsets_dev,
                                                     int32_t n_submeshes, const float* poses_dev,
                                                     float* world_vertices_dev, void* cuda_stream) {
  using namespace ags;
  if (!ctx) {
    set_error("ags_transform_vertices_noalloc: ctx is NULL");
    return AGS_ERR_INVALID_ARG;
  }
  if (n_vertices < 0 || n_submeshes < 0) {
    set_error("ags_transform_vertices_noalloc: negative size");
    return AGS_ERR_INVALID_ARG;
  }
  if (n_submeshes > kNoAllocMaxSubmeshes) {
    set_error("ags_transform_vertices_noalloc: n_submeshes exceeds the maximum of 65536 its fixed scratch holds");
    return AGS_ERR_INVALID_ARG;
  }
  if (n_vertices == 0) return AGS_OK;
  if (n_submeshes == 0 || !base_vertices_dev || !submesh_vertex_offsets_dev || !poses_dev || !world_vertices_dev) {
    set_error("ags_transform_vertices_noalloc: NULL pointer or vertices without sub-meshes");
    return AGS_ERR_INVALID_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(world_vertices_dev) & 15u) != 0) {
    set_error("ags_transform_vertices_noalloc: world_vertices_dev must be 16-byte aligned");
    return AGS_ERR_INVALID_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != ctx->device) {
    const cudaError_t se = cudaSetDevice(ctx->device);
    if (se != cudaSuccess) return cuda_fail(se, "ags_transform_vertices_noalloc: cudaSetDevice");
  }
  float* rot = nullptr;
  ags_status st = noalloc_scratch(ctx->device, &rot);
  if (st == AGS_OK) {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_submesh_rotations<<<blocks_for(n_submeshes, 128), 128, 0, s>>>(poses_dev, n_submeshes, rot);
    k_transform_vertices<<<blocks_for(n_vertices, 256), 256, 0, s>>>(base_vertices_dev, n_vertices,
                                                                     submesh_vertex_offsets_dev, n_submeshes, rot,
                                                                     poses_dev,
                                                                     reinterpret_cast<float4*>(world_vertices_dev));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "ags_transform_vertices_noalloc launch");
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return st;
}
