// Two-level scenes (AGS_BUILD_INSTANCED): every object (sub-mesh) gets its own
// BVH, built once in its own frame, and each environment a small BVH over the
// world-space boxes of its objects' parts (an object's root, or the children
// of the root of an object as large as its environment). Moving objects then
// only rebuilds the small top level and rewrites the object table; the object
// BVHs never change. This is
// one way to maintain the per-environment meshes M_{i,t} of Sec. III-D.1 as
// obstacles move; results equal a single-level scene's within float32
// rounding (the ray, not the mesh, is moved into each object's frame).
#include <cmath>
#include <memory>

#include "internal.cuh"

namespace ags {
namespace {

unsigned blocks_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// object table: world-to-object rotation R(q)^T, position, object BVH root, first triangle in its environment
__global__ void k_instances(const float* __restrict__ poses, int32_t J, const int32_t* __restrict__ obj_root,
                            const int32_t* __restrict__ tri_base, InstanceDev* __restrict__ inst) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  const float* P = poses + 7 * (int64_t)j;
  const float x = P[3], y = P[4], z = P[5], w = P[6];
  const float s = 2.0f / (x * x + y * y + z * z + w * w);
  InstanceDev d;
  // rows of R^T are the columns of R
  d.rt[0] = 1.0f - s * (y * y + z * z);
  d.rt[1] = s * (x * y + z * w);
  d.rt[2] = s * (x * z - y * w);
  d.rt[3] = s * (x * y - z * w);
  d.rt[4] = 1.0f - s * (x * x + z * z);
  d.rt[5] = s * (y * z + x * w);
  d.rt[6] = s * (x * z + y * w);
  d.rt[7] = s * (y * z - x * w);
  d.rt[8] = 1.0f - s * (x * x + y * y);
  d.p[0] = P[0];
  d.p[1] = P[1];
  d.p[2] = P[2];
  d.root = obj_root[j];
  d.tri_base = tri_base[j];
  d.pad[0] = d.pad[1] = 0;
  inst[j] = d;
}

// the root node of every object (an empty object: no slots)
__global__ void k_object_roots(const WideNode* __restrict__ nodes, const int32_t* __restrict__ root, int32_t J,
                               int64_t n_nodes, WideNode* __restrict__ out) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  const int32_t r = root[j];
  if (r >= 0 && r < n_nodes) {
    out[j] = nodes[r];
  } else {
    WideNode w{};
    w.child_base = -1;
    w.meta_lo = w.meta_hi = 0xFFFFFFFFu;
    out[j] = w;
  }
}

// the part table in the top level's leaf order
__global__ void k_parts_leaf_order(const int4* __restrict__ parts, const int32_t* __restrict__ leaf_tri, int32_t R,
                                   int32_t n_parts, int4* __restrict__ out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R) return;
  const int32_t t = leaf_tri[k];
  out[k] = (t >= 0 && t < n_parts) ? parts[t] : make_int4(-1, -1, 0, 0);
}

// The world box of object j at pose P: its object-frame box turned and moved
// in double precision, widened by 1e-5 of the coordinates (more than the
// float32 rounding of moving a ray into the object's frame).
void world_box(const double* ob, const float* P, double out[6]) {
  const double x = P[3], y = P[4], z = P[5], w = P[6];
  const double n = std::sqrt(x * x + y * y + z * z + w * w);
  const double qx = x / n, qy = y / n, qz = z / n, qw = w / n;
  const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw),     2 * (qx * qz + qy * qw),
                       2 * (qx * qy + qz * qw),     1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw),
                       2 * (qx * qz - qy * qw),     2 * (qy * qz + qx * qw),     1 - 2 * (qx * qx + qy * qy)};
  for (int a = 0; a < 3; ++a) {
    out[a] = INFINITY;
    out[3 + a] = -INFINITY;
  }
  double mag = 1.0;
  for (int c = 0; c < 8; ++c) {
    const double v[3] = {(c & 1) ? ob[3] : ob[0], (c & 2) ? ob[4] : ob[1], (c & 4) ? ob[5] : ob[2]};
    for (int a = 0; a < 3; ++a) {
      const double u = R[3 * a] * v[0] + R[3 * a + 1] * v[1] + R[3 * a + 2] * v[2] + P[a];
      out[a] = std::fmin(out[a], u);
      out[3 + a] = std::fmax(out[3 + a], u);
      mag = std::fmax(mag, std::fabs(u));
    }
  }
  for (int a = 0; a < 3; ++a) {
    out[a] -= 1e-5 * mag;
    out[3 + a] += 1e-5 * mag;
  }
}

// The top level: per environment, one degenerate "triangle" (lo, hi, lo) per
// part of its objects (an object's root, or the children of an opened root),
// whose box is the part's world box. One part per leaf slot, so every part is
// culled by its own box; the part table, put in the builder's leaf order,
// tells the render kernel which object and which node or leaf each is.
ags_status build_top(ags_context* ctx, const ags_scene* sc, const float* poses_h, ags_scene** out) {
  const int32_t E = sc->n_envs;
  const int64_t P = (int64_t)sc->h_parts.size();
  if (P > INT32_MAX / 4) {
    set_error("a two-level scene's top level holds at most 2^29 parts");
    return AGS_ERR_INVALID_ARG;
  }
  std::unique_ptr<ags_scene> top(new ags_scene());
  top->ctx = ctx;
  top->n_envs = E;
  top->n_tris = P;
  top->n_verts = 3 * P;
  top->flags = AGS_BVH_FP32 | AGS_SPLIT_CELLS(1) | AGS_LEAF_SIZE(1);
  top->env_tri_off.assign(E + 1, 0);
  top->env_vert_off.assign(E + 1, 0);
  top->env_sub_off.assign(E + 1, 0);
  std::vector<int32_t> sub_vert(1, 0), sub_env;
  std::vector<int64_t> sub_tri(1, 0);
  for (int32_t e = 0; e < E; ++e) {
    const int64_t n = sc->h_part_off[sc->env_sub_off[e + 1]] - sc->h_part_off[sc->env_sub_off[e]];
    top->env_tri_off[e + 1] = top->env_tri_off[e] + n;
    top->env_vert_off[e + 1] = top->env_vert_off[e] + 3 * n;
    top->env_sub_off[e + 1] = top->env_sub_off[e] + (n > 0 ? 1 : 0);
    if (n > 0) {
      sub_vert.push_back((int32_t)top->env_vert_off[e + 1]);
      sub_tri.push_back(top->env_tri_off[e + 1]);
      sub_env.push_back(e);
    }
  }
  const int64_t S = (int64_t)sub_env.size();
  top->n_subs = S;
  top->sub_tri_off = sub_tri;
  top->sub_seg.assign(S, 0);
  std::vector<float> verts(9 * P);
  std::vector<int32_t> vidx(3 * P);
  std::vector<int4> parts(std::max<int64_t>(P, 1));
  for (int64_t j = 0; j < sc->n_subs; ++j) {
    for (int64_t q = sc->h_part_off[j]; q < sc->h_part_off[j + 1]; ++q) {
      const ObjPart& pt = sc->h_parts[q];
      double b[6];
      world_box(pt.box, poses_h + 7 * j, b);
      const double c[9] = {b[0], b[1], b[2], b[3], b[4], b[5], b[0], b[1], b[2]};
      for (int k = 0; k < 9; ++k) {
        // round the low corner down and the high corner up
        float f = (float)c[k];
        const bool high = k >= 3 && k < 6;
        if (!high && (double)f > c[k]) f = std::nextafter(f, -INFINITY);
        if (high && (double)f < c[k]) f = std::nextafter(f, INFINITY);
        verts[9 * q + k] = f;
      }
      for (int k = 0; k < 3; ++k) vidx[3 * q + k] = (int32_t)(3 * q + k);
      parts[q] = make_int4((int32_t)j, pt.node, pt.leaf_start, pt.leaf_cnt);
    }
  }
  std::vector<float> ident(7 * std::max<int64_t>(S, 1), 0.0f);
  for (int64_t k = 0; k < S; ++k) ident[7 * k + 6] = 1.0f;
  ags_status st =
      build_scene(ctx, top.get(), verts.data(), vidx.data(), sub_vert.data(), ident.data(), sub_env.data());
  if (st == AGS_OK) {
    // the part table in leaf order (no splitting: one leaf reference per part)
    cudaStream_t s = ctx->stream;
    const int64_t R = top->n_refs;
    DevBufs tmp;
    int4* d_in = nullptr;
    cudaError_t e = tmp.alloc(&d_in, (size_t)std::max<int64_t>(P, 1));
    if (e == cudaSuccess) e = cudaMalloc(&top->d_parts, (size_t)std::max<int64_t>(R, 1) * sizeof(int4));
    if (e == cudaSuccess && P > 0)
      e = cudaMemcpyAsync(d_in, parts.data(), (size_t)P * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && R > 0) {
      k_parts_leaf_order<<<blocks_of(R, 256), 256, 0, s>>>(d_in, top->d.leaf_tri, (int32_t)R, (int32_t)P,
                                                           top->d_parts);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "two-level part table");
  }
  if (st != AGS_OK) {
    cudaStreamSynchronize(ctx->stream);
    cudaGetLastError();
    ags_scene_destroy(top.release());
    return st;
  }
  *out = top.release();
  return AGS_OK;
}

// Surface area of a box (lo xyz, hi xyz).
double box_area(const double* b) {
  const double x = std::fmax(b[3] - b[0], 0.0), y = std::fmax(b[4] - b[1], 0.0), z = std::fmax(b[5] - b[2], 0.0);
  return 2.0 * (x * y + y * z + z * x);
}

// An object whose world box has at least this fraction of its environment's
// box surface (a room's walls around everything else) is crossed by most of
// the environment's rays, and first, since its box holds the sensor; its root
// is opened into the top level, so that its children (the walls) become parts
// under their own boxes, culled and ordered like any other part. Opening the
// roots of the smaller objects too was measured slower (more parts, and a ray
// moved into the same object's frame once per part).
constexpr double kOpenAreaFraction = 0.25;

// The parts of every object: its root under the bounds of its vertices, or,
// for an opened root, each non-empty slot of the root (an inner child node or
// a leaf's triangle range) under the slot's float32 box.
ags_status object_parts(ags_context* ctx, ags_scene* sc, const float* poses_h) {
  cudaStream_t s = ctx->stream;
  const int32_t J = (int32_t)sc->n_subs;
  // world boxes of the objects and their environments at the build poses
  std::vector<double> wbox(6 * (size_t)std::max<int32_t>(J, 1));
  std::vector<double> env_area(std::max<int32_t>(J, 1), 0.0);
  for (int32_t e = 0; e < sc->n_envs; ++e) {
    double u[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int64_t j = sc->env_sub_off[e]; j < sc->env_sub_off[e + 1]; ++j) {
      world_box(&sc->h_obj_box[6 * j], poses_h + 7 * j, &wbox[6 * j]);
      if (sc->sub_tri_off[j + 1] == sc->sub_tri_off[j]) continue;
      for (int a = 0; a < 3; ++a) {
        u[a] = std::fmin(u[a], wbox[6 * j + a]);
        u[3 + a] = std::fmax(u[3 + a], wbox[6 * j + 3 + a]);
      }
    }
    for (int64_t j = sc->env_sub_off[e]; j < sc->env_sub_off[e + 1]; ++j) env_area[j] = box_area(u);
  }
  std::vector<WideNode> roots(std::max<int32_t>(J, 1));
  std::vector<int32_t> root_of(std::max<int32_t>(J, 1), -1);
  if (J > 0) {
    DevBufs tmp;
    WideNode* d_roots = nullptr;
    AGS_CHECK(tmp.alloc(&d_roots, (size_t)J));
    k_object_roots<<<blocks_of(J, 128), 128, 0, s>>>(static_cast<const WideNode*>(sc->objects->d.nodes),
                                                      sc->objects->d.env_root, J, sc->objects->n_nodes, d_roots);
    AGS_CHECK(cudaGetLastError());
    AGS_CHECK(cudaMemcpyAsync(roots.data(), d_roots, (size_t)J * sizeof(WideNode), cudaMemcpyDeviceToHost, s));
    AGS_CHECK(cudaMemcpyAsync(root_of.data(), sc->objects->d.env_root, (size_t)J * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, s));
    AGS_CHECK(cudaStreamSynchronize(s));
  }
  sc->h_parts.clear();
  sc->h_part_off.assign((size_t)J + 1, 0);
  for (int32_t j = 0; j < J; ++j) {
    const WideNode& w = roots[j];
    if (root_of[j] >= 0) {
      int slots = 0;
      for (int k = 0; k < 8; ++k)
        if ((((k < 4 ? w.meta_lo : w.meta_hi) >> (8 * (k & 3))) & 0xFFu) != kMetaEmpty) ++slots;
      if (slots > 1 && box_area(&wbox[6 * (size_t)j]) >= kOpenAreaFraction * env_area[j]) {
        const uint32_t b0 = w.meta_lo & 0xFFu;
        const int ni = (b0 & 0x80u) ? (int)std::min(b0 & 0xFu, 8u) : 0;
        for (int k = 0; k < 8; ++k) {
          const uint32_t m = ((k < 4 ? w.meta_lo : w.meta_hi) >> (8 * (k & 3))) & 0xFFu;
          if (m == kMetaEmpty) continue;
          ObjPart pt{};
          pt.box[0] = w.lox[k];
          pt.box[1] = w.loy[k];
          pt.box[2] = w.loz[k];
          pt.box[3] = w.hix[k];
          pt.box[4] = w.hiy[k];
          pt.box[5] = w.hiz[k];
          if (k < ni) {
            pt.node = w.child_base + k;
          } else {
            pt.node = -1;
            pt.leaf_start = w.tri_base + (int32_t)(m >> 2);
            pt.leaf_cnt = (int32_t)(m & 3u) + 1;
          }
          sc->h_parts.push_back(pt);
        }
      } else {
        ObjPart pt{};
        for (int a = 0; a < 6; ++a) pt.box[a] = sc->h_obj_box[6 * (int64_t)j + a];
        pt.node = root_of[j];
        sc->h_parts.push_back(pt);
      }
    }
    sc->h_part_off[j + 1] = (int64_t)sc->h_parts.size();
  }
  return AGS_OK;
}

// object table from host poses
ags_status write_instances(ags_context* ctx, ags_scene* sc, const float* poses_h) {
  cudaStream_t s = ctx->stream;
  const int32_t J = (int32_t)sc->n_subs;
  if (J == 0) return AGS_OK;
  DevBufs tmp;
  float* d_poses = nullptr;
  int32_t* d_base = nullptr;
  AGS_CHECK(tmp.alloc(&d_poses, 7 * (size_t)J));
  AGS_CHECK(tmp.alloc(&d_base, (size_t)J));
  std::vector<int32_t> base(J);
  for (int32_t e = 0; e < sc->n_envs; ++e)
    for (int64_t j = sc->env_sub_off[e]; j < sc->env_sub_off[e + 1]; ++j)
      base[j] = (int32_t)(sc->sub_tri_off[j] - sc->env_tri_off[e]);
  AGS_CHECK(cudaMemcpyAsync(d_poses, poses_h, 7 * (size_t)J * sizeof(float), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(d_base, base.data(), (size_t)J * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  k_instances<<<blocks_of(J, 128), 128, 0, s>>>(d_poses, J, sc->objects->d.env_root, d_base, sc->d_inst);
  AGS_CHECK(cudaGetLastError());
  // world vertices for read-back (ags_scene_get_world_triangles)
  ags_status st = transform_vertices(sc->d.base_verts, (int32_t)sc->n_verts, sc->d.sub_vert_off, J, d_poses,
                                     sc->d.world_verts, s);
  if (st != AGS_OK) return st;
  AGS_CHECK(cudaStreamSynchronize(s));
  return AGS_OK;
}

}  // namespace

ags_status build_instanced(ags_context* ctx, ags_scene* sc, const float* base_h, const int32_t* vidx_h,
                           const int32_t* sub_vert_h, const float* poses_h, const int32_t* sub_env_h) {
  (void)sub_env_h;
  cudaStream_t s = ctx->stream;
  const int32_t E = sc->n_envs;
  const int64_t J = sc->n_subs, V = sc->n_verts, F = sc->n_tris;
  if (J > 65536) {
    set_error("a two-level scene holds at most 65536 objects");
    return AGS_ERR_INVALID_ARG;
  }
  sc->node_format = kNodeFp32;
  // object level: one environment per object, in its own frame
  {
    std::unique_ptr<ags_scene> ob(new ags_scene());
    ob->ctx = ctx;
    ob->n_envs = (int32_t)std::max<int64_t>(J, 1);
    ob->n_tris = F;
    ob->n_verts = V;
    ob->n_subs = J;
    // no reference splitting within an object: its large triangles are not mixed with small ones from
    // other objects, and the split references only deepened each object's tree (15% slower renders)
    ob->flags = (sc->flags & ~(AGS_BUILD_INSTANCED | 0xFFu | (0xFFu << 12))) | AGS_SPLIT_CELLS(1);
    ob->env_tri_off.assign(ob->n_envs + 1, 0);
    ob->env_vert_off.assign(ob->n_envs + 1, 0);
    ob->env_sub_off.assign(ob->n_envs + 1, 0);
    for (int64_t j = 0; j < J; ++j) {
      ob->env_tri_off[j + 1] = sc->sub_tri_off[j + 1];
      ob->env_vert_off[j + 1] = sub_vert_h[j + 1];
      ob->env_sub_off[j + 1] = j + 1;
    }
    ob->sub_tri_off = sc->sub_tri_off;
    ob->sub_seg = sc->sub_seg;
    std::vector<float> ident(7 * std::max<int64_t>(J, 1), 0.0f);
    std::vector<int32_t> ob_env(std::max<int64_t>(J, 1));
    for (int64_t j = 0; j < J; ++j) {
      ident[7 * j + 6] = 1.0f;
      ob_env[j] = (int32_t)j;
    }
    ags_status st = build_scene(ctx, ob.get(), base_h, vidx_h, sub_vert_h, ident.data(), ob_env.data());
    if (st != AGS_OK) {
      cudaStreamSynchronize(s);
      ags_scene_destroy(ob.release());
      return st;
    }
    sc->objects = ob.release();
  }
  // object-frame boxes (from the vertices the objects' triangles use)
  sc->h_obj_box.assign(6 * J, 0.0);
  for (int64_t j = 0; j < J; ++j) {
    double* b = &sc->h_obj_box[6 * j];
    b[0] = b[1] = b[2] = INFINITY;
    b[3] = b[4] = b[5] = -INFINITY;
    for (int64_t t = sc->sub_tri_off[j]; t < sc->sub_tri_off[j + 1]; ++t)
      for (int c = 0; c < 3; ++c) {
        const float* v = base_h + 3 * (int64_t)vidx_h[3 * t + c];
        for (int a = 0; a < 3; ++a) {
          b[a] = std::fmin(b[a], (double)v[a]);
          b[3 + a] = std::fmax(b[3 + a], (double)v[a]);
        }
      }
    if (sc->sub_tri_off[j + 1] == sc->sub_tri_off[j])
      for (int a = 0; a < 6; ++a) b[a] = 0.0;  // an empty object: a point box, never entered below
  }
  // device copies: vertices (world read-back), object table, environment -> first object
  AGS_CHECK(cudaMalloc(&sc->d.base_verts, std::max<int64_t>(3 * V, 1) * sizeof(float)));
  AGS_CHECK(cudaMalloc(&sc->d.sub_vert_off, (size_t)(J + 1) * sizeof(int32_t)));
  AGS_CHECK(cudaMalloc(&sc->d.world_verts, std::max<int64_t>(V, 1) * sizeof(float4)));
  AGS_CHECK(cudaMalloc(&sc->d.tri_vidx, std::max<int64_t>(3 * F, 1) * sizeof(int32_t)));
  AGS_CHECK(cudaMalloc(&sc->d_inst, std::max<int64_t>(J, 1) * sizeof(InstanceDev)));
  AGS_CHECK(cudaMalloc(&sc->d_env_sub, (size_t)(E + 1) * sizeof(int32_t)));
  std::vector<int32_t> env_sub(E + 1);
  for (int32_t e = 0; e <= E; ++e) env_sub[e] = (int32_t)sc->env_sub_off[e];
  AGS_CHECK(cudaMemcpyAsync(sc->d.base_verts, base_h, 3 * (size_t)V * sizeof(float), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(sc->d.sub_vert_off, sub_vert_h, (size_t)(J + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                            s));
  AGS_CHECK(cudaMemcpyAsync(sc->d.tri_vidx, vidx_h, 3 * (size_t)F * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AGS_CHECK(cudaMemcpyAsync(sc->d_env_sub, env_sub.data(), (size_t)(E + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                            s));
  ags_status st = write_instances(ctx, sc, poses_h);
  if (st != AGS_OK) return st;
  if ((st = object_parts(ctx, sc, poses_h)) != AGS_OK) return st;
  if ((st = build_top(ctx, sc, poses_h, &sc->top)) != AGS_OK) return st;
  sc->n_nodes = sc->top->n_nodes + sc->objects->n_nodes;
  sc->n_refs = sc->objects->n_refs;
  sc->env_nodes = sc->top->env_nodes;
  return AGS_OK;
}

ags_status update_instanced(ags_context* ctx, ags_scene* sc, const float* poses_h) {
  NvtxRange range("ags two-level update");
  ags_scene* top = nullptr;
  ags_status st = build_top(ctx, sc, poses_h, &top);
  if (st != AGS_OK) return st;
  if ((st = write_instances(ctx, sc, poses_h)) != AGS_OK) {
    ags_scene_destroy(top);
    return st;
  }
  ags_scene_destroy(sc->top);
  sc->top = top;
  sc->n_nodes = sc->top->n_nodes + sc->objects->n_nodes;
  sc->env_nodes = sc->top->env_nodes;
  return AGS_OK;
}

void destroy_instanced(ags_scene* sc) {
  if (sc->objects) ags_scene_destroy(sc->objects);
  if (sc->top) ags_scene_destroy(sc->top);
  cudaFree(sc->d_inst);
  cudaFree(sc->d_env_sub);
  cudaFree(sc->d_parts);
  sc->objects = sc->top = nullptr;
  sc->d_inst = nullptr;
  sc->d_env_sub = nullptr;
  sc->d_parts = nullptr;
}

}  // namespace ags
