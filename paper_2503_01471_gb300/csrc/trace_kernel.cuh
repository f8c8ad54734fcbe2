// The render kernel, shared by the translation units that instantiate it.
// Batched ray casting (Sec. III-D.1: one ray per pixel tested against the
// environment's meshes M_{i,t}; range vs depth): one
// persistent launch over every environment's rays. Each warp repeatedly takes
// an 8x4 tile of pixels (env-major order, so one environment's BVH stays hot
// in L2 while all SMs work on it), generates the rays in registers, walks the
// environment's 8-wide BVH with a per-thread stack, tests leaf triangles with
// a watertight float32 test and writes depth/range and segment ID.
#pragma once
#include <cuda_fp16.h>

#include "internal.cuh"

namespace ags {

namespace {

constexpr int kTraceThreads = 128;
// optional work of the render kernel (template bits)
constexpr int kExtraChannels = 1;  // face index, barycentrics, normal, sensor-frame point
constexpr int kExtraShadow = 2;    // stereo shadow test towards a second sensor
constexpr int kExtraTable = 4;     // sensor-frame directions from a caller's table
#ifndef AGS_TRACE_MIN_BLOCKS
#define AGS_TRACE_MIN_BLOCKS 7
#endif
constexpr int kTraceMinBlocks = AGS_TRACE_MIN_BLOCKS;  // resident blocks per SM the register budget targets
constexpr int kStackSize = 64;
// Box culling is made conservative against float32 rounding: each slab
// bound is computed as one fma with a per-ray constant that already moves
// the near bound down and the far bound up by more than the rounding of
// -o/d, the slab exit is scaled up by (1 + 4u) and the current nearest hit by
// (1 + 2^-12), so a box holding the eventual nearest triangle is never skipped.
constexpr float kSlabSlack = 1.0f + 4.0f * 5.96046448e-8f;
constexpr float kCullSlack = 1.0f + 2.44140625e-4f;
constexpr float kSlabEps = 4.0f * 5.96046448e-8f;

struct Ray {
  float ix, iy, iz;          // 1 / direction
  float cnx, cny, cnz;       // near-bound constants: -o/d, lowered
  float cfx, cfy, cfz;       // far-bound constants: -o/d, raised
  int onx, ony, onz;         // float4 offsets of the near-bound arrays in a node (octant)
  // the inverse direction and the near / far constants again, each held twice as a register pair for the
  // packed arithmetic of the float32 node test (two children per instruction)
  float2 ix2, iy2, iz2, cnx2, cfx2, cny2, cfy2, cnz2, cfz2;
  // the watertight test's constants, in this thread's slot of shared memory (three float4: the rows of the
  // shear that maps v - o to the ray's frame, each with one origin coordinate in w). They are read only by
  // triangle tests, so keeping them out of registers leaves the traversal more registers.
  float4* frame;
};

__device__ __forceinline__ float nonzero(float d) {
  // an exactly-zero direction component is replaced by a tiny one of the same
  // sign for both the box and the triangle test, keeping them consistent
  return fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d;
}

// Packed FP32 arithmetic of Blackwell (fma / add / mul .rn.f32x2, sm_100 and later): one instruction
// performs two IEEE round-to-nearest operations, the same as two scalar __fmaf_rn / __fmul_rn, bit for bit.
// The node test applies them to two children at once.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// The ray o + t d: its slab constants in registers and (kTri) its
// triangle-test constants in r.frame, which the caller points at the
// thread's slot. A ray that only meets boxes skips the latter.
template <bool kTri = true>
__device__ __forceinline__ void setup_ray(Ray& r, float ox, float oy, float oz, float dx, float dy, float dz) {
  dx = nonzero(dx);
  dy = nonzero(dy);
  dz = nonzero(dz);
  r.ix = 1.0f / dx;
  r.iy = 1.0f / dy;
  r.iz = 1.0f / dz;
  const float px = -ox * r.ix, py = -oy * r.iy, pz = -oz * r.iz;
  const float ex = kSlabEps * fabsf(px), ey = kSlabEps * fabsf(py), ez = kSlabEps * fabsf(pz);
  r.cnx = px - ex;
  r.cfx = px + ex;
  r.cny = py - ey;
  r.cfy = py + ey;
  r.cnz = pz - ez;
  r.cfz = pz + ez;
  // node layout (float4 units): header, lox[2], hix[2], loy[2], hiy[2], loz[2], hiz[2]
  r.ix2 = make_float2(r.ix, r.ix);
  r.iy2 = make_float2(r.iy, r.iy);
  r.iz2 = make_float2(r.iz, r.iz);
  r.cnx2 = make_float2(r.cnx, r.cnx);
  r.cfx2 = make_float2(r.cfx, r.cfx);
  r.cny2 = make_float2(r.cny, r.cny);
  r.cfy2 = make_float2(r.cfy, r.cfy);
  r.cnz2 = make_float2(r.cnz, r.cnz);
  r.cfz2 = make_float2(r.cfz, r.cfz);
  r.onx = r.ix >= 0.0f ? 1 : 3;
  r.ony = r.iy >= 0.0f ? 5 : 7;
  r.onz = r.iz >= 0.0f ? 9 : 11;
  if (!kTri) return;
  // watertight shear: z axis = largest |d| component, x/y the next two in
  // cyclic order (swapped when d_z < 0 to keep the winding)
  const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
  const int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  const float dkz = kz == 0 ? dx : (kz == 1 ? dy : dz);
  if (dkz < 0.0f) {
    const int t = kx;
    kx = ky;
    ky = t;
  }
  const float dkx = kx == 0 ? dx : (kx == 1 ? dy : dz);
  const float dky = ky == 0 ? dx : (ky == 1 ? dy : dz);
  const float Sx = dkx / dkz, Sy = dky / dkz, Sz = 1.0f / dkz;
  r.frame[0] = make_float4((kx == 0 ? 1.0f : 0.0f) - (kz == 0 ? Sx : 0.0f),
                           (kx == 1 ? 1.0f : 0.0f) - (kz == 1 ? Sx : 0.0f),
                           (kx == 2 ? 1.0f : 0.0f) - (kz == 2 ? Sx : 0.0f), ox);
  r.frame[1] = make_float4((ky == 0 ? 1.0f : 0.0f) - (kz == 0 ? Sy : 0.0f),
                           (ky == 1 ? 1.0f : 0.0f) - (kz == 1 ? Sy : 0.0f),
                           (ky == 2 ? 1.0f : 0.0f) - (kz == 2 ? Sy : 0.0f), oy);
  r.frame[2] = make_float4(kz == 0 ? Sz : 0.0f, kz == 1 ? Sz : 0.0f, kz == 2 ? Sz : 0.0f, oz);
}

// Watertight ray/triangle test (Woop, Benthin, Wald 2013), two-sided with
// closed edges. Each vertex is sheared by the same per-ray rows (so a vertex
// shared by two triangles gets the same coordinates in both), and each edge
// function is an explicitly rounded difference of two rounded products, so a
// shared edge gives exactly opposite values in its two triangles and no ray
// slips between them.
__device__ __forceinline__ void shear(const float4* f, const float4 v, float& X, float& Y, float& Z) {
  const float ax = __fsub_rn(v.x, f[0].w), ay = __fsub_rn(v.y, f[1].w), az = __fsub_rn(v.z, f[2].w);
  X = __fmaf_rn(f[0].x, ax, __fmaf_rn(f[0].y, ay, __fmul_rn(f[0].z, az)));
  Y = __fmaf_rn(f[1].x, ax, __fmaf_rn(f[1].y, ay, __fmul_rn(f[1].z, az)));
  Z = __fmaf_rn(f[2].x, ax, __fmaf_rn(f[2].y, ay, __fmul_rn(f[2].z, az)));
}

template <bool kChannels>
__device__ __forceinline__ void test_triangle(const Ray& r, const float4* __restrict__ tris, int32_t k,
                                              float& t_best, int32_t& best_id, int32_t& best_seg, int32_t& best_k) {
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
  // reject t < 0, and |t| beyond the current best (with slack) before dividing
  if (T != 0.0f && ((__float_as_uint(T) ^ __float_as_uint(det)) >> 31)) return;
  const float aT = fabsf(T), adet = fabsf(det);
  if (aT > t_best * adet * kCullSlack) return;
  const float t = __fdiv_rn(aT, adet);
  const int32_t id = __float_as_int(b.w);
  if (t < t_best || (t == t_best && id < best_id)) {
    t_best = t;
    best_id = id;
    best_seg = __float_as_int(a.w);
    if constexpr (kChannels) best_k = k;
  }
}

// Barycentric weights (of the second and third vertex) of the ray's hit on
// packed triangle k: the edge functions of the watertight test, recomputed
// with the same operations, over their sum.
__device__ __forceinline__ void hit_barycentrics(const Ray& r, const float4* __restrict__ tris, int32_t k, float& u,
                                                 float& v) {
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
  const float det = U + V + W;
  u = __fdiv_rn(V, det);
  v = __fdiv_rn(W, det);
}

// Unit geometric normal (b - a) x (c - a) of packed triangle k, turned to
// face the ray (direction d).
__device__ __forceinline__ void hit_normal(const float4* __restrict__ tris, int32_t k, float dx, float dy, float dz,
                                           float& nx, float& ny, float& nz) {
  const float4 a = __ldg(tris + 3 * (int64_t)k);
  const float4 b = __ldg(tris + 3 * (int64_t)k + 1);
  const float4 c = __ldg(tris + 3 * (int64_t)k + 2);
  // explicitly rounded, so that every kernel variant gives the same bits
  const float e1x = __fsub_rn(b.x, a.x), e1y = __fsub_rn(b.y, a.y), e1z = __fsub_rn(b.z, a.z);
  const float e2x = __fsub_rn(c.x, a.x), e2y = __fsub_rn(c.y, a.y), e2z = __fsub_rn(c.z, a.z);
  nx = __fmaf_rn(e1y, e2z, -__fmul_rn(e1z, e2y));
  ny = __fmaf_rn(e1z, e2x, -__fmul_rn(e1x, e2z));
  nz = __fmaf_rn(e1x, e2y, -__fmul_rn(e1y, e2x));
  float s = rsqrtf(__fmaf_rn(nz, nz, __fmaf_rn(ny, ny, __fmul_rn(nx, nx))));
  if (__fmaf_rn(nz, dz, __fmaf_rn(ny, dy, __fmul_rn(nx, dx))) > 0.0f) s = -s;
  nx = __fmul_rn(nx, s);
  ny = __fmul_rn(ny, s);
  nz = __fmul_rn(nz, s);
}

// ---- one wide node: header, and per child the entry distance and whether
// the ray's slab interval meets [0, t_cull]. Every bound t = b * ix + c is a
// single fma whose constant is already lowered (near) or raised (far) by more
// than the rounding of c. Children k and k+1 are tested together: their slab
// distances come in register pairs (packed arithmetic), and one packed
// multiply scales both exits up by the slack.
__device__ __forceinline__ void child_test2(int k, float2 tnx, float2 tfx, float2 tny, float2 tfy, float2 tnz,
                                            float2 tfz, float t_cull, float* tmins, uint32_t& hit_mask) {
  const float tmin0 = max3f(tnx.x, tny.x, fmaxf(tnz.x, 0.0f)), tmin1 = max3f(tnx.y, tny.y, fmaxf(tnz.y, 0.0f));
  const float2 tmax = mul2(make_float2(min3f(tfx.x, tfy.x, tfz.x), min3f(tfx.y, tfy.y, tfz.y)),
                           make_float2(kSlabSlack, kSlabSlack));
  tmins[k] = tmin0;
  tmins[k + 1] = tmin1;
  if (tmin0 <= fminf(tmax.x, t_cull)) hit_mask |= 1u << k;
  if (tmin1 <= fminf(tmax.y, t_cull)) hit_mask |= 2u << k;
}

// near / far constants of one axis for a node whose bounds are origin + b:
// c = (origin - o) / d, computed as one fma from the ray's lowered / raised
// constants, then moved away again by the rounding of that fma
__device__ __forceinline__ void node_axis(float origin, float inv, float cn_ray, float cf_ray, float& cn, float& cf) {
  const float n = __fmaf_rn(origin, inv, cn_ray), f = __fmaf_rn(origin, inv, cf_ray);
  cn = n - kSlabEps * fabsf(n);
  cf = f + kSlabEps * fabsf(f);
}

template <int kFmt>
__device__ __forceinline__ void test_node(const void* __restrict__ nodes, int32_t node, const Ray& r, float t_cull,
                                          int32_t& child_base, int32_t& tri_base, uint32_t& meta_lo,
                                          uint32_t& meta_hi, float* tmins, uint32_t& hit_mask) {
  hit_mask = 0;
  if constexpr (kFmt == kNodeFp32) {
    const float4* np = reinterpret_cast<const float4*>(nodes) + (int64_t)node * 13;
    const float4 h = __ldg(np);
    child_base = __float_as_int(h.x);
    tri_base = __float_as_int(h.y);
    meta_lo = __float_as_uint(h.z);
    meta_hi = __float_as_uint(h.w);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const float4 nx4 = __ldg(np + r.onx + half), fx4 = __ldg(np + (4 - r.onx) + half);
      const float4 ny4 = __ldg(np + r.ony + half), fy4 = __ldg(np + (12 - r.ony) + half);
      const float4 nz4 = __ldg(np + r.onz + half), fz4 = __ldg(np + (20 - r.onz) + half);
      const float nxs[4] = {nx4.x, nx4.y, nx4.z, nx4.w}, fxs[4] = {fx4.x, fx4.y, fx4.z, fx4.w};
      const float nys[4] = {ny4.x, ny4.y, ny4.z, ny4.w}, fys[4] = {fy4.x, fy4.y, fy4.z, fy4.w};
      const float nzs[4] = {nz4.x, nz4.y, nz4.z, nz4.w}, fzs[4] = {fz4.x, fz4.y, fz4.z, fz4.w};
#pragma unroll
      for (int q = 0; q < 4; q += 2) {
        // children q, q+1 of this half: adjacent words of one 16-byte load form each register pair
        const float2 tnx = fma2(make_float2(nxs[q], nxs[q + 1]), r.ix2, r.cnx2);
        const float2 tfx = fma2(make_float2(fxs[q], fxs[q + 1]), r.ix2, r.cfx2);
        const float2 tny = fma2(make_float2(nys[q], nys[q + 1]), r.iy2, r.cny2);
        const float2 tfy = fma2(make_float2(fys[q], fys[q + 1]), r.iy2, r.cfy2);
        const float2 tnz = fma2(make_float2(nzs[q], nzs[q + 1]), r.iz2, r.cnz2);
        const float2 tfz = fma2(make_float2(fzs[q], fzs[q + 1]), r.iz2, r.cfz2);
        child_test2(4 * half + q, tnx, tfx, tny, tfy, tnz, tfz, t_cull, tmins, hit_mask);
      }
    }
  } else if constexpr (kFmt == kNodeFp16) {
    // 128 B: header, origin, then lo_x, hi_x, lo_y, hi_y, lo_z, hi_z as 8 halves each
    const float4* np = reinterpret_cast<const float4*>(nodes) + (int64_t)node * 8;
    const float4 h = __ldg(np), org = __ldg(np + 1);
    child_base = __float_as_int(h.x);
    tri_base = __float_as_int(h.y);
    meta_lo = __float_as_uint(h.z);
    meta_hi = __float_as_uint(h.w);
    float cnx, cfx, cny, cfy, cnz, cfz;
    node_axis(org.x, r.ix, r.cnx, r.cfx, cnx, cfx);
    node_axis(org.y, r.iy, r.cny, r.cfy, cny, cfy);
    node_axis(org.z, r.iz, r.cnz, r.cfz, cnz, cfz);
    const int sx = (r.onx >> 1) & 1, sy = (r.ony >> 1) & 1, sz = (r.onz >> 1) & 1;  // 1: negative direction
    const float4 nx = __ldg(np + 2 + sx), fx = __ldg(np + 3 - sx);
    const float4 ny = __ldg(np + 4 + sy), fy = __ldg(np + 5 - sy);
    const float4 nz = __ldg(np + 6 + sz), fz = __ldg(np + 7 - sz);
    const float nxw[4] = {nx.x, nx.y, nx.z, nx.w}, fxw[4] = {fx.x, fx.y, fx.z, fx.w};
    const float nyw[4] = {ny.x, ny.y, ny.z, ny.w}, fyw[4] = {fy.x, fy.y, fy.z, fy.w};
    const float nzw[4] = {nz.x, nz.y, nz.z, nz.w}, fzw[4] = {fz.x, fz.y, fz.z, fz.w};
    const float2 cnx2 = make_float2(cnx, cnx), cfx2 = make_float2(cfx, cfx), cny2 = make_float2(cny, cny),
                 cfy2 = make_float2(cfy, cfy), cnz2 = make_float2(cnz, cnz), cfz2 = make_float2(cfz, cfz);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      // the two halves of a word are children 2w and 2w+1
      const float2 bnx = __half22float2(*reinterpret_cast<const __half2*>(&nxw[w]));
      const float2 bfx = __half22float2(*reinterpret_cast<const __half2*>(&fxw[w]));
      const float2 bny = __half22float2(*reinterpret_cast<const __half2*>(&nyw[w]));
      const float2 bfy = __half22float2(*reinterpret_cast<const __half2*>(&fyw[w]));
      const float2 bnz = __half22float2(*reinterpret_cast<const __half2*>(&nzw[w]));
      const float2 bfz = __half22float2(*reinterpret_cast<const __half2*>(&fzw[w]));
      child_test2(2 * w, fma2(bnx, r.ix2, cnx2), fma2(bfx, r.ix2, cfx2), fma2(bny, r.iy2, cny2),
                  fma2(bfy, r.iy2, cfy2), fma2(bnz, r.iz2, cnz2), fma2(bfz, r.iz2, cfz2), t_cull, tmins, hit_mask);
    }
  } else {
    // 80 B: origin + per-axis power-of-two scale exponents, header, then per
    // axis 8 low and 8 high 8-bit bounds: bound = origin + q * 2^(e - 127)
    const float4* np = reinterpret_cast<const float4*>(nodes) + (int64_t)node * 5;
    const float4 org = __ldg(np), h = __ldg(np + 1);
    child_base = __float_as_int(h.x);
    tri_base = __float_as_int(h.y);
    meta_lo = __float_as_uint(h.z);
    meta_hi = __float_as_uint(h.w);
    const uint32_t ex = __float_as_uint(org.w);
    const float scx = __uint_as_float((ex & 0xFFu) << 23), scy = __uint_as_float(((ex >> 8) & 0xFFu) << 23),
                scz = __uint_as_float(((ex >> 16) & 0xFFu) << 23);
    float cnx, cfx, cny, cfy, cnz, cfz;
    node_axis(org.x, r.ix, r.cnx, r.cfx, cnx, cfx);
    node_axis(org.y, r.iy, r.cny, r.cfy, cny, cfy);
    node_axis(org.z, r.iz, r.cnz, r.cfz, cnz, cfz);
    const float ax = scx * r.ix, ay = scy * r.iy, az = scz * r.iz;  // exact: powers of two
    const int sx = (r.onx >> 1) & 1, sy = (r.ony >> 1) & 1, sz = (r.onz >> 1) & 1;
    const uint4 qx = __ldg(reinterpret_cast<const uint4*>(np + 2));
    const uint4 qy = __ldg(reinterpret_cast<const uint4*>(np + 3));
    const uint4 qz = __ldg(reinterpret_cast<const uint4*>(np + 4));
    // near words: lo (x, y) for a positive direction, hi (z, w) for a negative one
    const uint32_t nx0 = sx ? qx.z : qx.x, nx1 = sx ? qx.w : qx.y, fx0 = sx ? qx.x : qx.z, fx1 = sx ? qx.y : qx.w;
    const uint32_t ny0 = sy ? qy.z : qy.x, ny1 = sy ? qy.w : qy.y, fy0 = sy ? qy.x : qy.z, fy1 = sy ? qy.y : qy.w;
    const uint32_t nz0 = sz ? qz.z : qz.x, nz1 = sz ? qz.w : qz.y, fz0 = sz ? qz.x : qz.z, fz1 = sz ? qz.y : qz.w;
    // children k, k+1 together (packed arithmetic, as for float32 nodes)
    const float2 ax2 = make_float2(ax, ax), ay2 = make_float2(ay, ay), az2 = make_float2(az, az);
    const float2 cnx2 = make_float2(cnx, cnx), cfx2 = make_float2(cfx, cfx), cny2 = make_float2(cny, cny),
                 cfy2 = make_float2(cfy, cfy), cnz2 = make_float2(cnz, cnz), cfz2 = make_float2(cfz, cfz);
    const float2 m23 = make_float2(-8388608.0f, -8388608.0f);
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      // bytes k, k+1 of the word as exact floats q: bits 0x4B000000 | q = 2^23 + q, less 2^23
      auto q2 = [&](uint32_t w0, uint32_t w1) {
        const uint32_t w = k < 4 ? w0 : w1;
        return add2(make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | (uint32_t)(k & 3))),
                                __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | (uint32_t)((k + 1) & 3)))),
                    m23);
      };
      child_test2(k, fma2(q2(nx0, nx1), ax2, cnx2), fma2(q2(fx0, fx1), ax2, cfx2), fma2(q2(ny0, ny1), ay2, cny2),
                  fma2(q2(fy0, fy1), ay2, cfy2), fma2(q2(nz0, nz1), az2, cnz2), fma2(q2(fz0, fz1), az2, cfz2), t_cull,
                  tmins, hit_mask);
    }
  }
}

// Any-hit test of packed triangle k against the segment o + t d, t in
// [t0, t1] (the same watertight arithmetic as test_triangle).
__device__ __forceinline__ bool segment_hits(const Ray& r, const float4* __restrict__ tris, int32_t k, float t0,
                                             float t1) {
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
  if (neg && pos) return false;
  const float det = U + V + W;
  if (det == 0.0f) return false;
  const float T = __fmaf_rn(U, Az, __fmaf_rn(V, Bz, __fmul_rn(W, Cz)));
  if (T != 0.0f && ((__float_as_uint(T) ^ __float_as_uint(det)) >> 31)) return false;
  const float t = __fdiv_rn(fabsf(T), fabsf(det));
  return t >= t0 && t <= t1;
}

// Stereo shadow (Sec. III-D.1): does any triangle of environment env meet
// the segment o + t d, t in [t0, t1]? The caller casts it from the second
// sensor towards the hit P (o = o2, d = P - o2, t in [0, 1 - eps]): the same
// segment as from P back to the sensor, but every ray of a warp starts at
// the same point, which keeps the warp's traversals alike. The traversal
// stops at the first such triangle; children are visited in slot order.
// Limits set the status word and `failed`.
template <int kFmt>
__device__ bool occluded(const TraceArgs& a, int32_t env, float px, float py, float pz, float dx, float dy, float dz,
                         float t0, float t1, int2* stack, float4* frame, bool& failed) {
  Ray r;
  r.frame = frame;
  setup_ray(r, px, py, pz, dx, dy, dz);
  int32_t node = __ldg(a.env_root + env);
  int sp = 0, visits = 0;
  const float t_cull = kCullSlack;
  while (node >= 0) {
    if (++visits > a.max_visits) {
      atomicOr(a.status, kStatusIterationCap);
      failed = true;
      return false;
    }
    if (node >= a.n_nodes) {
      atomicOr(a.status, kStatusBadIndex);
      failed = true;
      return false;
    }
    int32_t child_base, tri_base;
    uint32_t meta_lo, meta_hi, hit_mask;
    float tmins[8];
    test_node<kFmt>(a.nodes, node, r, t_cull, child_base, tri_base, meta_lo, meta_hi, tmins, hit_mask);
    const uint32_t b0 = meta_lo & 0xFFu;
    const int ni = (b0 & 0x80u) ? (int)min(b0 & 0xFu, 8u) : 0;
    const uint32_t inner_bits = (1u << ni) - 1u;
    uint32_t leaf_mask = hit_mask & ~inner_bits;
    uint32_t inner_hits = hit_mask & inner_bits;
    while (leaf_mask) {
      const int k = __ffs(leaf_mask) - 1;
      leaf_mask &= leaf_mask - 1;
      const uint32_t m = ((k < 4 ? meta_lo : meta_hi) >> (8 * (k & 3))) & 0xFFu;
      if (m == kMetaEmpty) continue;
      const int32_t start = tri_base + (int32_t)(m >> 2);
      const int32_t cnt = (int32_t)(m & 3u) + 1;
      if (start < 0 || start + cnt > a.n_tris) {
        atomicOr(a.status, kStatusBadIndex);
        failed = true;
        return false;
      }
      for (int32_t x = 0; x < cnt; ++x)
        if (segment_hits(r, a.tris, start + x, t0, t1)) return true;
    }
    node = -1;
    if (inner_hits) {
      node = child_base + (__ffs(inner_hits) - 1);
      inner_hits &= inner_hits - 1;
      while (inner_hits) {
        if (sp >= kStackSize) {
          atomicOr(a.status, kStatusStackOverflow);
          failed = true;
          return false;
        }
        stack[sp++] = make_int2(child_base + (__ffs(inner_hits) - 1), 0);
        inner_hits &= inner_hits - 1;
      }
    } else if (sp > 0) {
      node = stack[--sp].x;
    }
  }
  return false;
}

// a3: the sensor-frame direction of pixel / beam (row, col). Camera: the
// unnormalised (1, a, b) through the pixel centre, so the distance along it
// is the depth itself; LiDAR: the unit beam direction (distance = range);
// ray table: the caller's row as given (distance in units of its length).
template <bool kTable>
__device__ __forceinline__ void sensor_dir(const SensorParams& sen, int32_t row, int32_t col, float& lx, float& ly,
                                           float& lz) {
  if constexpr (kTable) {
    const float* g = sen.dirs + 3 * ((int64_t)row * sen.W + col);
    lx = __ldg(g);
    ly = __ldg(g + 1);
    lz = __ldg(g + 2);
  } else if (sen.type == AGS_PINHOLE) {
    lx = 1.0f;
    ly = __fmul_rn(0.5f * (float)sen.W - ((float)col + 0.5f), sen.inv_f);  // the difference is exact
    lz = __fmul_rn(0.5f * (float)sen.H - ((float)row + 0.5f), sen.inv_f);
  } else {
    float sin_el, cos_el, sin_az, cos_az;
    sincosf(__fmaf_rn(-(float)row, sen.dv, sen.vmax), &sin_el, &cos_el);
    sincosf(__fmul_rn(sen.hfov, __fdiv_rn((float)col, (float)sen.W)), &sin_az, &cos_az);
    lx = __fmul_rn(cos_el, cos_az);
    ly = __fmul_rn(cos_el, sin_az);
    lz = sin_el;
  }
}

template <bool kSlots>
__device__ __forceinline__ const float* slot_pose(const TraceArgs& a, int32_t slot) {
  if constexpr (kSlots) return a.slots[slot].pose;
  else return a.poses + 7 * (int64_t)slot;
}
template <bool kSlots>
__device__ __forceinline__ int64_t slot_out(const TraceArgs& a, const SensorParams& sen, int32_t slot) {
  if constexpr (kSlots) return __ldg(&a.slots[slot].out_offset);
  else return (int64_t)slot * sen.H * sen.W;
}

// One step of a ray's nearest-hit traversal (a4-a6): test the eight children
// of `node`, the triangles of its hit leaves (they tighten t_best before any
// descent), then pick the next node: the nearest hit inner child (the
// others pushed, farthest deepest), else the nearest stacked node still
// within the cull distance. Returns -1 when the ray is done; sets `failed`
// (and the status word) on an out-of-range triangle range or a full stack.
template <bool kCount, int kFmt, bool kChannels, int kStack = kStackSize>
__device__ __forceinline__ int32_t visit_node(const TraceArgs& a, const Ray& r, int32_t node, float& t_best,
                                              int32_t& best_id, int32_t& best_seg, int32_t& best_k, int2* stack,
                                              int& sp, bool& failed, unsigned long long& n_tris) {
  int32_t* __restrict__ status = a.status;
  const float t_cull = t_best * kCullSlack;
  int32_t child_base, tri_base;
  uint32_t meta_lo, meta_hi;
  float tmins[8];
  uint32_t hit_mask;
  test_node<kFmt>(a.nodes, node, r, t_cull, child_base, tri_base, meta_lo, meta_hi, tmins, hit_mask);
  const uint32_t b0 = meta_lo & 0xFFu;
  const int ni = (b0 & 0x80u) ? (int)min(b0 & 0xFu, 8u) : 0;
  const uint32_t inner_bits = (1u << ni) - 1u;
  uint32_t leaf_mask = hit_mask & ~inner_bits;
  const uint32_t inner_hits = hit_mask & inner_bits;
  // leaves of this node first: they tighten t_best before descending
  while (leaf_mask) {
    const int k = __ffs(leaf_mask) - 1;
    leaf_mask &= leaf_mask - 1;
    const uint32_t m = ((k < 4 ? meta_lo : meta_hi) >> (8 * (k & 3))) & 0xFFu;
    if (m == kMetaEmpty) continue;
    const int32_t start = tri_base + (int32_t)(m >> 2);
    const int32_t cnt = (int32_t)(m & 3u) + 1;
    if (start < 0 || start + cnt > a.n_tris) {
      atomicOr(status, kStatusBadIndex);
      failed = true;
      return -1;
    }
    for (int32_t x = 0; x < cnt; ++x)
      test_triangle<kChannels>(r, a.tris, start + x, t_best, best_id, best_seg, best_k);
    if (kCount) n_tris += cnt;
  }
  const int n_inner = __popc(inner_hits);
  if (n_inner == 1) return child_base + (__ffs(inner_hits) - 1);  // the common case: no ordering needed
  if (n_inner == 2) {
    // two children: the nearer is taken, the farther pushed (keys: tmin bits, slot in the low 3 bits); their
    // entry distances picked out by slot with selects (keeping tmins in registers)
    const int k1 = __ffs(inner_hits) - 1, k2 = 31 - __clz(inner_hits);
    float t1 = tmins[0], t2 = tmins[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      t1 = k == k1 ? tmins[k] : t1;
      t2 = k == k2 ? tmins[k] : t2;
    }
    const uint32_t key1 = (__float_as_uint(t1) & ~7u) | (uint32_t)k1;
    const uint32_t key2 = (__float_as_uint(t2) & ~7u) | (uint32_t)k2;
    const uint32_t kmin = min(key1, key2), kfar = max(key1, key2);
    const uint32_t key_cull = __float_as_uint(t_best * kCullSlack);
    if ((kfar & ~7u) <= key_cull) {
      if (sp >= kStack) {
        // the full stack reports an overflow; a short one marks the ray for the full-stack retry pass
        if (kStack == kStackSize) atomicOr(status, kStatusStackOverflow);
        else sp = kStack + 1;
        failed = true;
        return -1;
      }
      stack[sp++] = make_int2(child_base + (int32_t)(kfar & 7u), (int32_t)(kfar & ~7u));
    }
    if ((kmin & ~7u) <= key_cull) return child_base + (int32_t)(kmin & 7u);
  } else if (n_inner > 1) {
    // nearest first (sorting network on keys: tmin bits with the slot in the low 3 bits)
    uint32_t keys[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      keys[k] = ((inner_hits >> k) & 1u) ? ((__float_as_uint(tmins[k]) & ~7u) | (uint32_t)k) : 0xFFFFFFFFu;
#define AGS_CSWAP(i, j)                         \
  {                                             \
  const uint32_t lo_ = min(keys[i], keys[j]); \
  const uint32_t hi_ = max(keys[i], keys[j]); \
  keys[i] = lo_;                              \
  keys[j] = hi_;                              \
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
        if (sp >= kStack) {
          if (kStack == kStackSize) atomicOr(status, kStatusStackOverflow);
          else sp = kStack + 1;
          failed = true;
        } else {
          stack[sp++] = make_int2(child_base + (int32_t)(keys[k] & 7u), (int32_t)(keys[k] & ~7u));
        }
      }
    }
    if (failed) return -1;
    if ((keys[0] & ~7u) <= key_cull) return child_base + (int32_t)(keys[0] & 7u);
  }
  const float t_pop = t_best * kCullSlack;
  while (sp > 0) {
    const int2 e = stack[--sp];
    if (__int_as_float(e.y) <= t_pop) return e.x;
  }
  return -1;
}

// The rotation R(q) (rows R[0..8]) of the sensor pose P = (p, q), q
// normalised. Every operation is explicitly rounded, so the compiler has no
// freedom to fuse a multiply and an add differently in different kernels:
// every kernel variant casts exactly the same rays. False for a pose the
// method cannot use (q near zero, or anything non-finite).
__device__ __forceinline__ bool pose_rotation(const float* P, float* R) {
  const float px = __ldg(P), py = __ldg(P + 1), pz = __ldg(P + 2);
  const float qx = __ldg(P + 3), qy = __ldg(P + 4), qz = __ldg(P + 5), qw = __ldg(P + 6);
  const float n2 = __fmaf_rn(qw, qw, __fmaf_rn(qz, qz, __fmaf_rn(qy, qy, __fmul_rn(qx, qx))));
  if (!(n2 >= 1e-30f) || !isfinite(n2) || !isfinite(__fadd_rn(__fadd_rn(px, py), pz))) return false;
  const float s = __fdiv_rn(2.0f, n2);
  const float xx = __fmul_rn(qx, qx), yy = __fmul_rn(qy, qy), zz = __fmul_rn(qz, qz);
  R[0] = __fmaf_rn(-s, __fadd_rn(yy, zz), 1.0f);
  R[4] = __fmaf_rn(-s, __fadd_rn(xx, zz), 1.0f);
  R[8] = __fmaf_rn(-s, __fadd_rn(xx, yy), 1.0f);
  R[1] = __fmul_rn(s, __fmaf_rn(qx, qy, -__fmul_rn(qz, qw)));
  R[3] = __fmul_rn(s, __fmaf_rn(qx, qy, __fmul_rn(qz, qw)));
  R[2] = __fmul_rn(s, __fmaf_rn(qx, qz, __fmul_rn(qy, qw)));
  R[6] = __fmul_rn(s, __fmaf_rn(qx, qz, -__fmul_rn(qy, qw)));
  R[5] = __fmul_rn(s, __fmaf_rn(qy, qz, -__fmul_rn(qx, qw)));
  R[7] = __fmul_rn(s, __fmaf_rn(qy, qz, __fmul_rn(qx, qw)));
  return true;
}

// R l for sensor-frame l, explicitly rounded.
__device__ __forceinline__ void rotate(const float* R, float lx, float ly, float lz, float& dx, float& dy,
                                       float& dz) {
  dx = __fmaf_rn(R[2], lz, __fmaf_rn(R[1], ly, __fmul_rn(R[0], lx)));
  dy = __fmaf_rn(R[5], lz, __fmaf_rn(R[4], ly, __fmul_rn(R[3], lx)));
  dz = __fmaf_rn(R[8], lz, __fmaf_rn(R[7], ly, __fmul_rn(R[6], lx)));
}

// a3: the world ray of pixel / beam (row, col) from the sensor pose P =
// (p, q): origin p, direction R(q) l with l the sensor-frame direction, and
// R itself. False for a pose or table row the method cannot use. The same
// bits whether l comes from the camera model (lx = 1 folded) or a table.
template <bool kTable>
__device__ __forceinline__ bool make_ray(const SensorParams& sen, const float* P, int32_t row, int32_t col, Ray& r,
                                         float* R, float& lx, float& ly, float& lz) {
  if (!pose_rotation(P, R)) return false;
  sensor_dir<kTable>(sen, row, col, lx, ly, lz);
  if (kTable && (!isfinite(lx + ly + lz) || (lx == 0.0f && ly == 0.0f && lz == 0.0f))) return false;
  float dx, dy, dz;
  rotate(R, lx, ly, lz, dx, dy, dz);
  setup_ray(r, __ldg(P), __ldg(P + 1), __ldg(P + 2), dx, dy, dz);
  return true;
}

// a6: the reported value and segment of a finished ray (failed: NaN, -1).
__device__ __forceinline__ void resolve_hit(const SensorParams& sen, bool failed, float t_best, int32_t best_id,
                                            int32_t best_seg, float& v, int32_t& seg) {
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
}

// a4-a6 for one ray: the nearest-hit walk of environment env's BVH from its
// root. On return `failed` says whether a limit stopped it; with a short
// stack (kStack < kStackSize), sp == kStack + 1 says the stack ran out.
template <bool kCount, int kFmt, bool kChannels, int kStack>
__device__ __forceinline__ void walk_ray(const TraceArgs& a, const Ray& r, int32_t env, float& t_best,
                                         int32_t& best_id, int32_t& best_seg, int32_t& best_k, int2* stack, int& sp,
                                         bool& failed, unsigned long long& n_nodes, unsigned long long& n_tris) {
  int32_t* __restrict__ status = a.status;
  int32_t node = __ldg(a.env_root + env);
  int visits = 0;
  sp = 0;
  failed = false;
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
    node = visit_node<kCount, kFmt, kChannels, kStack>(a, r, node, t_best, best_id, best_seg, best_k, stack, sp,
                                                       failed, n_tris);
    if (failed) break;
  }
}

// The rays of one warp tile: sensor shape `sen`, environment `env`, tile
// index t_in within it; `slot` locates the pose and the outputs (the
// environment's index in the launch, or the request's slot in the table).
// A short stack (kStack < kStackSize, plain renders only) hands each ray
// that outgrows it to the retry list, which k_trace_retry walks again with
// the full stack; such a ray writes no output here.
template <bool kCount, int kTileW, int kRaysPerLane, bool kSlots, int kFmt, int kExtra, int kStack = kStackSize>
__device__ __forceinline__ void trace_tile(const TraceArgs& a, const SensorParams& sen, int32_t env, int32_t t_in,
                                           int32_t slot, int lane, int2* stack, float4* frames,
                                           unsigned long long& n_nodes, unsigned long long& n_tris,
                                           unsigned long long& n_rays) {
  constexpr int kTileH = 32 * kRaysPerLane / kTileW;
  int32_t* __restrict__ status = a.status;
  const int32_t tile_x0 = (t_in % sen.tiles_x) * kTileW;
  const int32_t tile_y0 = (t_in / sen.tiles_x) * kTileH;

  for (int rr = 0; rr < kRaysPerLane; ++rr) {
  const int idx = rr * 32 + lane;
  const int32_t col = tile_x0 + (idx % kTileW);
  const int32_t row = tile_y0 + (idx / kTileW);
  const int32_t W = sen.W, H = sen.H;
  if (col >= W || row >= H) continue;

  // ---- a3: ray generation from the sensor pose (p, q); recomputed per ray
  // (L1-resident) so that nothing of it stays live during the traversal
  const float* P = slot_pose<kSlots>(a, slot);
  Ray r;
  r.frame = frames;
  float R[9], lx, ly, lz;
  if (!make_ray<(kExtra & kExtraTable) != 0>(sen, P, row, col, r, R, lx, ly, lz)) {
    // a pose (or table row) the method cannot use: flag it and report NaN for this ray
    atomicOr(status, kStatusBadPose);
    if (!kCount) {
      const int64_t o = slot_out<kSlots>(a, sen, slot) + (int64_t)row * W + col;
      a.out_depth[o] = __int_as_float(0x7fc00000);
      a.out_seg[o] = -1;
    }
    continue;
  }

  // ---- a4-a6: traversal, triangle tests, nearest hit
  float t_best = sen.max_range;  // camera: depth limit; LiDAR: range limit (unit direction)
  int32_t best_id = 0x7fffffff, best_seg = -1, best_k = -1;
  int sp;
  bool failed;
  walk_ray<kCount, kFmt, (kExtra & kExtraChannels) != 0, kStack>(a, r, env, t_best, best_id, best_seg, best_k, stack,
                                                                  sp, failed, n_nodes, n_tris);

  if (kCount) {
    ++n_rays;
    continue;
  }
  if constexpr (kStack < kStackSize) {
    if (sp > kStack) {
      // the short stack ran out: the full-stack retry pass renders this ray
      const unsigned int i = atomicAdd(a.retry_count, 1u);
      if (i < (unsigned int)a.retry_cap) {
        a.retry_list[i] = slot_out<kSlots>(a, sen, slot) + (int64_t)row * W + col;
        continue;
      }
      atomicOr(status, kStatusStackOverflow);  // the retry list is full: reported like an overflow
    }
  }
  float v;
  int32_t seg;
  resolve_hit(sen, failed, t_best, best_id, best_seg, v, seg);
  if constexpr ((kExtra & kExtraShadow) != 0) {
    if (!failed && seg >= 0) {
      // the hit point P and the second sensor o2 = p + R b, both in the world
      float sx, sy, sz;
      sensor_dir<(kExtra & kExtraTable) != 0>(sen, row, col, sx, sy, sz);
      float dwx, dwy, dwz, bwx, bwy, bwz;
      rotate(R, sx, sy, sz, dwx, dwy, dwz);
      rotate(R, a.baseline[0], a.baseline[1], a.baseline[2], bwx, bwy, bwz);
      const float px = frames[0].w, py = frames[1].w, pz = frames[2].w;
      const float Px = __fmaf_rn(t_best, dwx, px), Py = __fmaf_rn(t_best, dwy, py), Pz = __fmaf_rn(t_best, dwz, pz);
      const float o2x = __fadd_rn(px, bwx), o2y = __fadd_rn(py, bwy), o2z = __fadd_rn(pz, bwz);
      bool sfail = false;
      const bool shadowed = occluded<kFmt>(a, env, o2x, o2y, o2z, __fsub_rn(Px, o2x), __fsub_rn(Py, o2y),
                                           __fsub_rn(Pz, o2z), 0.0f, __fsub_rn(1.0f, a.shadow_eps), stack,
                                           frames + 3, sfail);
      if (sfail) {
        failed = true;
        v = __int_as_float(0x7fc00000);
        seg = -1;
      } else if (shadowed) {
        v = sen.max_range;
        seg = -1;
      }
    }
  }
  const int64_t o = slot_out<kSlots>(a, sen, slot) + (int64_t)row * W + col;
  a.out_depth[o] = v;
  a.out_seg[o] = seg;
  if constexpr ((kExtra & kExtraChannels) != 0) {
    // extra hit channels of the reported hit (a miss or a near hit reported
    // as invalid: face -1, zero weights and normal)
    const float nan = __int_as_float(0x7fc00000);
    int32_t face = failed ? -1 : (seg >= 0 ? best_id : -1);
    float bu = failed ? nan : 0.0f, bv = bu, nx = bu, ny = bu, nz = bu;
    if (face >= 0 && best_k >= 0) {
      hit_barycentrics(r, a.tris, best_k, bu, bv);
      hit_normal(a.tris, best_k, __frcp_rn(r.ix), __frcp_rn(r.iy), __frcp_rn(r.iz), nx, ny, nz);
    }
    if (a.out_face) a.out_face[o] = face;
    if (a.out_bary) {
      a.out_bary[2 * o] = bu;
      a.out_bary[2 * o + 1] = bv;
    }
    if (a.out_normal) {
      a.out_normal[3 * o] = nx;
      a.out_normal[3 * o + 1] = ny;
      a.out_normal[3 * o + 2] = nz;
    }
    if (a.out_point) {
      // the hit in the sensor frame: reported value along the sensor-frame direction
      sensor_dir<(kExtra & kExtraTable) != 0>(sen, row, col, lx, ly, lz);
      a.out_point[3 * o] = __fmul_rn(v, lx);
      a.out_point[3 * o + 1] = __fmul_rn(v, ly);
      a.out_point[3 * o + 2] = __fmul_rn(v, lz);
    }
  }
  }  // rays of this lane in the tile
}

// The persistent tile loop of the render kernels: each warp takes tiles from
// the global counter until none is left.
template <bool kCount, int kTileW, int kRaysPerLane, bool kSlots, int kFmt, int kExtra, int kStack>
__device__ __forceinline__ void run_tiles(const TraceArgs& a) {
  const int lane = threadIdx.x & 31;
  int2 stack[kStack];
  // each thread's slot for its ray's triangle-test constants (a second one for the stereo shadow ray)
  constexpr int kFrames = (kExtra & kExtraShadow) ? 2 : 1;
  __shared__ float4 s_frames[kTraceThreads * 3 * kFrames];
  float4* frames = s_frames + 3 * kFrames * threadIdx.x;
  unsigned long long n_nodes = 0, n_tris = 0, n_rays = 0;
  int64_t total_tiles = a.total_tiles;
  int32_t n_slots = a.n_slots;
  if constexpr (kSlots) {
    // a batch replayed from a captured graph carries its size in device memory
    if (a.slot_header) {
      n_slots = __ldg(a.slot_header);
      total_tiles = __ldg(a.slot_header + 1);
    }
  }

  while (true) {
    unsigned int tile = 0;
    if (lane == 0) tile = atomicAdd(a.tile_counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if ((int64_t)tile >= total_tiles) break;
    int32_t env, t_in, slot, slot_spec = 0;
    if constexpr (kSlots) {
      // the slot holding this tile: last slot whose first tile is <= tile
      int32_t lo = 0, hi = n_slots - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if ((unsigned)__ldg(&a.slots[mid].tile_begin) <= tile) lo = mid; else hi = mid - 1;
      }
      slot = lo;
      env = __ldg(&a.slots[lo].env);
      slot_spec = __ldg(&a.slots[lo].spec);
      if ((unsigned)slot_spec >= (unsigned)a.n_specs) {
        if (lane == 0) atomicOr(a.status, kStatusBadIndex);
        continue;
      }
      t_in = (int32_t)(tile - (unsigned)__ldg(&a.slots[lo].tile_begin));
    } else {
      slot = (int32_t)(tile / (unsigned)a.sensor.tiles_per_env);
      t_in = (int32_t)(tile - (unsigned)slot * (unsigned)a.sensor.tiles_per_env);
      env = a.env_ids ? __ldg(a.env_ids + slot) : slot;
    }
    if ((unsigned)env >= (unsigned)a.n_scene_envs) {
      if (lane == 0) atomicOr(a.status, kStatusBadIndex);
      continue;
    }
    if constexpr (kSlots) {
      trace_tile<kCount, kTileW, kRaysPerLane, true, kFmt, kExtra, kStack>(a, a.specs[slot_spec], env, t_in, slot,
                                                                           lane, stack, frames, n_nodes, n_tris,
                                                                           n_rays);
    } else {
      trace_tile<kCount, kTileW, kRaysPerLane, false, kFmt, kExtra, kStack>(a, a.sensor, env, t_in, slot, lane,
                                                                            stack, frames, n_nodes, n_tris, n_rays);
    }
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

// kSlots: each tile belongs to one slot of a table (serving: every request has
// its own environment, sensor shape, pose and output offset); otherwise all
// environments of the launch share one sensor shape.
template <bool kCount, int kTileW, int kRaysPerLane, bool kSlots, int kFmt, int kExtra = 0>
__global__ void __launch_bounds__(kTraceThreads, kTraceMinBlocks) k_trace(const TraceArgs a) {
  run_tiles<kCount, kTileW, kRaysPerLane, kSlots, kFmt, kExtra, kStackSize>(a);
}

// The plain render (8x4 tiles) with a kStack-entry stack; rays that need more
// go to the retry list (a short stack is a tuning choice: results are those
// of the full stack).
template <int kFmt, int kStack>
__global__ void __launch_bounds__(kTraceThreads, kTraceMinBlocks) k_trace_short(const TraceArgs a) {
  run_tiles<false, 8, 1, false, kFmt, 0, kStack>(a);
}

// The retry pass after k_trace_short: one thread per listed ray, walked with
// the full stack, output written as k_trace would.
template <int kFmt>
__global__ void __launch_bounds__(kTraceThreads, kTraceMinBlocks) k_trace_retry(const TraceArgs a) {
  const SensorParams& sen = a.sensor;
  const unsigned int n = min(*a.retry_count, (unsigned int)a.retry_cap);
  const int64_t per = (int64_t)sen.W * sen.H;
  int2 stack[kStackSize];
  __shared__ float4 s_frames[kTraceThreads * 3];
  unsigned long long no_count = 0;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int64_t o = a.retry_list[i];
    const int32_t slot = (int32_t)(o / per);
    const int32_t pix = (int32_t)(o - (int64_t)slot * per);
    const int32_t row = pix / sen.W, col = pix - row * sen.W;
    const int32_t env = a.env_ids ? __ldg(a.env_ids + slot) : slot;
    Ray r;
    r.frame = s_frames + 3 * threadIdx.x;
    float R[9], lx, ly, lz;
    if (slot < 0 || slot >= a.n || (unsigned)env >= (unsigned)a.n_scene_envs ||
        !make_ray<false>(sen, a.poses + 7 * (int64_t)slot, row, col, r, R, lx, ly, lz)) {
      atomicOr(a.status, kStatusBadIndex);  // the first pass listed only rays it could cast
      continue;
    }
    float t_best = sen.max_range;
    int32_t best_id = 0x7fffffff, best_seg = -1, best_k = -1;
    int sp;
    bool failed;
    walk_ray<false, kFmt, false, kStackSize>(a, r, env, t_best, best_id, best_seg, best_k, stack, sp, failed, no_count,
                                             no_count);
    float v;
    int32_t seg;
    resolve_hit(sen, failed, t_best, best_id, best_seg, v, seg);
    a.out_depth[o] = v;
    a.out_seg[o] = seg;
  }
}

}  // namespace

}  // namespace ags
