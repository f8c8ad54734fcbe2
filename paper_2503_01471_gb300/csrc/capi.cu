// C ABI of the renderer (include/ags.h): argument validation, context and
// scene lifetime, kernel launches. No torch types, no exceptions across the
// boundary; every failure is an ags_status plus a thread-local message.
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "internal.cuh"

namespace ags {

// brute.cu: every triangle copy of each ray's environment, no tree (a test aid). env_ref_dev and
// env_tri_dev are the [E+1] reference and triangle offsets, leaf_tri_dev the [R] input triangle of each
// leaf-order copy; temp holds brute_temp_bytes(R) bytes.
cudaError_t launch_brute(const TraceArgs& a, const int32_t* env_ref_dev, const int32_t* env_tri_dev,
                         const int32_t* leaf_tri_dev, int32_t E, int32_t R, void* temp, cudaStream_t s);
size_t brute_temp_bytes(int32_t R);

SensorParams sensor_params(const ags_sensor_spec* spec, int tile_w, int tile_h) {
  SensorParams p;
  p.W = spec->width;
  p.H = spec->height;
  p.type = spec->type;
  p.near_mode = spec->near_mode;
  p.inv_f = (float)(std::tan(0.5 * (double)spec->hfov_rad) / (0.5 * (double)spec->width));
  p.hfov = spec->hfov_rad;
  p.vmax = spec->vfov_max_rad;
  p.dv = spec->height > 1 ? (float)(((double)spec->vfov_max_rad - (double)spec->vfov_min_rad) / (spec->height - 1))
                          : 0.0f;
  p.min_range = spec->min_range;
  p.max_range = spec->max_range;
  p.tiles_x = (spec->width + tile_w - 1) / tile_w;
  p.tiles_per_env = p.tiles_x * ((spec->height + tile_h - 1) / tile_h);
  p.dirs = nullptr;
  return p;
}

namespace {
thread_local std::string g_last_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ags_status invalid(const std::string& msg) {
  set_error(msg);
  return AGS_ERR_INVALID_ARG;
}

bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

ags_status check_spec(const ags_sensor_spec* s, bool with_table) {
  if (!s) return invalid("spec is NULL");
  if (s->type == AGS_RAY_TABLE && !with_table) return invalid("AGS_RAY_TABLE sensors render through ags_render_ex");
  if (s->type != AGS_RAY_TABLE && with_table) return invalid("a ray table needs an AGS_RAY_TABLE sensor");
  if (s->type != AGS_PINHOLE && s->type != AGS_LIDAR && s->type != AGS_RAY_TABLE)
    return invalid("spec.type must be AGS_PINHOLE, AGS_LIDAR or AGS_RAY_TABLE");
  if (s->width < 1 || s->width > 16384 || s->height < 1 || s->height > 16384)
    return invalid("spec.width/height must be in [1, 16384]");
  if (!std::isfinite(s->min_range) || !std::isfinite(s->max_range) || s->min_range < 0.0f ||
      !(s->max_range > s->min_range))
    return invalid("spec ranges must satisfy 0 <= min_range < max_range < inf");
  if (s->near_mode != AGS_NEAR_CLAMP && s->near_mode != AGS_NEAR_INVALID) return invalid("spec.near_mode invalid");
  if (s->flags != 0) return invalid("spec.flags must be 0");
  const double pi = 3.14159265358979323846;
  if (s->type == AGS_PINHOLE) {
    if (!(s->hfov_rad > 0.0f) || !(s->hfov_rad < (float)pi)) return invalid("camera hfov must be in (0, pi)");
  } else if (s->type == AGS_LIDAR) {
    if (!(s->hfov_rad > 0.0f) || !(s->hfov_rad <= (float)(2.0 * pi) + 1e-6f))
      return invalid("LiDAR azimuth span must be in (0, 2 pi]");
    if (!std::isfinite(s->vfov_min_rad) || !std::isfinite(s->vfov_max_rad) || s->vfov_min_rad < -(float)(pi / 2) - 1e-6f ||
        s->vfov_max_rad > (float)(pi / 2) + 1e-6f || s->vfov_min_rad > s->vfov_max_rad)
      return invalid("LiDAR elevations must satisfy -pi/2 <= vfov_min <= vfov_max <= pi/2");
  }
  return AGS_OK;
}

unsigned int* tile_counter(ags_context* ctx, cudaStream_t s) {
  auto it = ctx->tile_counters.find(s);
  if (it != ctx->tile_counters.end()) return it->second;
  unsigned int* p = nullptr;
  if (cudaMalloc(&p, sizeof(unsigned int)) != cudaSuccess) return nullptr;
  ctx->tile_counters[s] = p;
  return p;
}

ags_launch_config default_config() { return {8, 1, 0, 0.0f, 0}; }

ags_launch_config lookup_config(const ags_scene* sc, const ags_sensor_spec* spec) {
  auto it = sc->launch.find({spec->type, spec->width, spec->height});
  return it != sc->launch.end() ? it->second : default_config();
}

int max_blocks_per_sm(ags_context* ctx) { return ctx->sm_count > 0 ? ctx->trace_blocks / ctx->sm_count : 1; }

ags_status check_config(ags_context* ctx, const ags_launch_config* c) {
  if (!c) return invalid("launch config is NULL");
  if (!trace_shape_supported(c->tile_w, c->rays_per_lane))
    return invalid("unsupported launch shape: (tile_w, rays_per_lane) must be one of (8,1) (4,1) (16,1) (32,1) "
                   "(8,2) (16,2) (16,4)");
  if (c->blocks_per_sm < 0 || c->blocks_per_sm > max_blocks_per_sm(ctx))
    return invalid("blocks_per_sm must be 0 .. the kernel's occupancy limit");
  if (c->stack_depth != 0 && c->stack_depth != 16 && c->stack_depth != 32 && c->stack_depth != 64)
    return invalid("stack_depth must be 0 (64), 16, 32 or 64");
  if ((c->stack_depth == 16 || c->stack_depth == 32) && (c->tile_w != 8 || c->rays_per_lane != 1))
    return invalid("a short stack (16 or 32) renders with the 8x4 tile");
  return AGS_OK;
}

ags_status fill_trace_args(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, int32_t n,
                           const int32_t* env_ids, const float* poses, float* depth, int32_t* seg, TraceArgs& a,
                           const ags_launch_config& cfg) {
  if (sc->objects) {
    // two levels: the top level walks like a scene, the objects below it
    if (cfg.tile_w != 8 || cfg.rays_per_lane != 1) return invalid("two-level scenes render with the 8x4 tile");
    a.nodes = sc->top->d.nodes;
    a.node_format = kNodeFp32;
    a.tris = sc->top->d.tris;
    a.env_root = sc->top->d.env_root;
    a.n_nodes = (int32_t)sc->top->n_nodes;
    a.n_tris = (int32_t)sc->top->n_refs;
    a.instanced = 1;
    a.inst = sc->d_inst;
    a.n_inst = (int32_t)sc->n_subs;
    a.env_sub = sc->d_env_sub;
    a.obj_nodes = sc->objects->d.nodes;
    a.obj_tris = sc->objects->d.tris;
    a.obj_n_nodes = (int32_t)sc->objects->n_nodes;
    a.obj_n_tris = (int32_t)sc->objects->n_refs;
    a.parts = sc->top->d_parts;
  } else {
    a.nodes = sc->d.nodes;
    a.node_format = sc->node_format;
    a.tris = sc->d.tris;
    a.env_root = sc->d.env_root;
    a.n_nodes = (int32_t)sc->n_nodes;
    a.n_tris = (int32_t)sc->n_refs;
  }
  a.n_scene_envs = sc->n_envs;
  a.env_ids = env_ids;
  a.poses = poses;
  a.out_depth = depth;
  a.out_seg = seg;
  a.n = n;
  int lw = 0;
  while ((1 << lw) < cfg.tile_w) ++lw;
  a.log2_tile_w = lw;
  a.rays_per_lane = cfg.rays_per_lane;
  a.stack_depth = (sc->objects || cfg.stack_depth == 0) ? 64 : cfg.stack_depth;
  a.retry_list = ctx->d_retry_list;
  a.retry_count = ctx->d_retry_count;
  a.retry_cap = ctx->retry_cap;
  a.tile_h = 32 * cfg.rays_per_lane / cfg.tile_w;
  a.sensor = sensor_params(spec, cfg.tile_w, a.tile_h);
  int64_t total = (int64_t)a.sensor.tiles_per_env * n;
  if (total >= (1ll << 31)) return invalid("too many rays in one render call (tiles >= 2^31)");
  a.total_tiles = total;
  a.status = ctx->d_status;
  a.counts = ctx->d_counts;
  a.max_visits = ctx->max_node_visits;
  return AGS_OK;
}

ags_status launch(ags_context* ctx, TraceArgs& a, cudaStream_t s, bool count, int blocks_per_sm = 0) {
  NvtxRange range(count ? "ags render (count)" : "ags render");
  unsigned int* counter = tile_counter(ctx, s);
  if (!counter) {
    set_error("cannot allocate the tile counter");
    return AGS_ERR_OUT_OF_MEMORY;
  }
  a.tile_counter = counter;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(tile counter)");
  if (a.total_tiles == 0) return AGS_OK;
  const int blocks = count ? ctx->trace_count_blocks
                           : (blocks_per_sm > 0 ? ctx->sm_count * blocks_per_sm : ctx->trace_blocks);
  if (!count && a.stack_depth < 64 && !a.slots && !a.extra && !a.instanced) {
    // short stack: its overflows go to the retry list, walked again with the full stack
    e = cudaMemsetAsync(a.retry_count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(retry count)");
    e = launch_trace_short(a, blocks, ctx->sm_count * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_trace_short launch");
    return AGS_OK;
  }
  e = launch_trace(a, blocks, count, s);
  if (e != cudaSuccess) return cuda_fail(e, "k_trace launch");
  return AGS_OK;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

ags_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? AGS_ERR_OUT_OF_MEMORY : AGS_ERR_CUDA;
}

}  // namespace ags

using namespace ags;

#define AGS_API_BEGIN try {
#define AGS_API_END                                   \
  }                                                   \
  catch (const std::bad_alloc&) {                     \
    set_error("host allocation failed");              \
    return AGS_ERR_OUT_OF_MEMORY;                     \
  }                                                   \
  catch (...) {                                       \
    set_error("unexpected host exception");           \
    return AGS_ERR_CUDA;                              \
  }

extern "C" {

const char* ags_last_error(void) { return g_last_error.c_str(); }

ags_status ags_context_create(int device, ags_context** out) {
  AGS_API_BEGIN
  if (!out) return invalid("out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return invalid("device index out of range");
  DeviceGuard g(device);
  ags_context* ctx = new ags_context();
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->d_status, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&ctx->d_counts, 3 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&ctx->d_retry_list, (size_t)kRetryAlloc * sizeof(int64_t))) != cudaSuccess ||
      (e = cudaMalloc(&ctx->d_retry_count, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMemset(ctx->d_status, 0, sizeof(int))) != cudaSuccess) {
    ags_status st = cuda_fail(e, "context setup");
    ags_context_destroy(ctx);
    return st;
  }
  ctx->retry_cap = kRetryAlloc;
  ctx->trace_blocks = ctx->sm_count * trace_blocks_per_sm(false);
  ctx->trace_count_blocks = ctx->sm_count * trace_blocks_per_sm(true);
  *out = ctx;
  return AGS_OK;
  AGS_API_END
}

void ags_context_destroy(ags_context* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->tile_counters) cudaFree(kv.second);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_counts);
  cudaFree(ctx->d_retry_list);
  cudaFree(ctx->d_retry_count);
  cudaFree(ctx->stage);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

ags_status ags_context_set_traversal_cap(ags_context* ctx, int32_t max_node_visits) {
  if (!ctx) return invalid("ctx is NULL");
  if (max_node_visits < 1) return invalid("max_node_visits must be >= 1");
  ctx->max_node_visits = max_node_visits;
  return AGS_OK;
}

ags_status ags_context_set_retry_capacity(ags_context* ctx, int32_t rays) {
  if (!ctx) return invalid("ctx is NULL");
  if (rays < 0 || rays > kRetryAlloc) return invalid("rays must be in [0, 1048576]");
  ctx->retry_cap = rays;
  return AGS_OK;
}

ags_status ags_scene_build(ags_context* ctx, const ags_env_mesh* envs, int32_t n_envs, const float* obstacle_poses,
                           uint32_t build_flags, ags_scene** out) {
  AGS_API_BEGIN
  if (!out) return invalid("out is NULL");
  *out = nullptr;
  if (!ctx) return invalid("ctx is NULL");
  if (!envs) return invalid("envs is NULL");
  if (n_envs < 1 || n_envs > 65536) return invalid("n_envs must be in [1, 65536]");
  if ((build_flags & 0xFFu) > AGS_BVH_Q8) return invalid("unsupported BVH node format in build_flags");
  if ((build_flags & ~(0xFFFFFu | AGS_BUILD_LBVH | AGS_BUILD_INSTANCED | AGS_BUILD_GREEDY_COLLAPSE |
                       AGS_CLUSTER_RADIUS(128))) != 0)
    return invalid("unknown bits in build_flags");
  if ((build_flags & AGS_BUILD_INSTANCED) && (build_flags & 0xFFu) != AGS_BVH_FP32)
    return invalid("two-level scenes use float32 nodes");
  if (((build_flags >> 8) & 0xFu) > (uint32_t)kMaxLeafTris) return invalid("leaf size must be 1..4");
  // sizes
  int64_t J = 0, V = 0, F = 0;
  for (int32_t e = 0; e < n_envs; ++e) {
    if (envs[e].n_submeshes < 0) return invalid("env " + std::to_string(e) + ": n_submeshes < 0");
    if (envs[e].n_submeshes > 0 && !envs[e].submeshes) return invalid("env " + std::to_string(e) + ": submeshes NULL");
    for (int32_t j = 0; j < envs[e].n_submeshes; ++j) {
      const ags_submesh& m = envs[e].submeshes[j];
      if (m.n_vertices < 0 || m.n_triangles < 0)
        return invalid("env " + std::to_string(e) + " submesh " + std::to_string(j) + ": negative size");
      V += m.n_vertices;
      F += m.n_triangles;
    }
    J += envs[e].n_submeshes;
  }
  if (F >= (1ll << 31) - 1 || V >= (1ll << 31) - 1 || J >= (1ll << 31) - 1)
    return invalid("scene too large (2^31 - 1 triangles, vertices or sub-meshes)");
  if (J > 0 && !obstacle_poses) return invalid("obstacle_poses is NULL");

  std::unique_ptr<ags_scene> sc(new ags_scene());
  sc->ctx = ctx;
  sc->n_envs = n_envs;
  sc->n_tris = F;
  sc->n_verts = V;
  sc->n_subs = J;
  sc->flags = build_flags;
  sc->env_tri_off.assign(n_envs + 1, 0);
  sc->env_vert_off.assign(n_envs + 1, 0);
  sc->env_sub_off.assign(n_envs + 1, 0);
  sc->sub_tri_off.assign(J + 1, 0);
  sc->sub_seg.assign(J, 0);
  std::vector<float> base(3 * V);
  std::vector<int32_t> vidx(3 * F), sub_vert(J + 1, 0), sub_env(J);
  int64_t j_all = 0, v_all = 0, f_all = 0;
  for (int32_t e = 0; e < n_envs; ++e) {
    for (int32_t j = 0; j < envs[e].n_submeshes; ++j, ++j_all) {
      const ags_submesh& m = envs[e].submeshes[j];
      std::string where = "env " + std::to_string(e) + " submesh " + std::to_string(j);
      if (m.n_vertices > 0 && !m.vertices) return invalid(where + ": vertices NULL");
      if (m.n_triangles > 0 && !m.indices) return invalid(where + ": indices NULL");
      if (m.segment_id < 0) return invalid(where + ": segment_id < 0");
      for (int32_t v = 0; v < m.n_vertices; ++v)
        if (!finite3(m.vertices + 3 * (int64_t)v)) return invalid(where + ": non-finite vertex");
      for (int64_t k = 0; k < 3 * (int64_t)m.n_triangles; ++k) {
        int32_t x = m.indices[k];
        if (x < 0 || x >= m.n_vertices) return invalid(where + ": triangle index out of range");
        vidx[3 * f_all + k] = (int32_t)v_all + x;
      }
      const float* p = obstacle_poses + 7 * j_all;
      for (int k = 0; k < 7; ++k)
        if (!std::isfinite(p[k])) return invalid(where + ": non-finite pose");
      double qn = (double)p[3] * p[3] + (double)p[4] * p[4] + (double)p[5] * p[5] + (double)p[6] * p[6];
      if (!(qn > 1e-12) || !std::isfinite(qn)) return invalid(where + ": quaternion has zero length");
      if (m.n_vertices > 0) std::memcpy(base.data() + 3 * v_all, m.vertices, 3 * (size_t)m.n_vertices * sizeof(float));
      sub_env[j_all] = e;
      sc->sub_seg[j_all] = m.segment_id;
      v_all += m.n_vertices;
      f_all += m.n_triangles;
      sub_vert[j_all + 1] = (int32_t)v_all;
      sc->sub_tri_off[j_all + 1] = f_all;
    }
    sc->env_tri_off[e + 1] = f_all;
    sc->env_vert_off[e + 1] = v_all;
    sc->env_sub_off[e + 1] = j_all;
  }
  DeviceGuard g(ctx->device);
  ags_status st = (build_flags & AGS_BUILD_INSTANCED)
                      ? build_instanced(ctx, sc.get(), base.data(), vidx.data(), sub_vert.data(), obstacle_poses,
                                        sub_env.data())
                      : build_scene(ctx, sc.get(), base.data(), vidx.data(), sub_vert.data(), obstacle_poses,
                                    sub_env.data());
  if (st == AGS_OK) {
    sc->h_base = std::move(base);
    sc->h_vidx = std::move(vidx);
    sc->h_sub_vert = std::move(sub_vert);
    sc->h_sub_env = std::move(sub_env);
    if (J > 0) sc->h_poses.assign(obstacle_poses, obstacle_poses + 7 * J);
  }
  if (st != AGS_OK) {
    cudaStreamSynchronize(ctx->stream);
    ags_scene_destroy(sc.release());
    cudaGetLastError();  // a failed allocation must not surface in a later call
    return st;
  }
  *out = sc.release();
  return AGS_OK;
  AGS_API_END
}

void ags_scene_destroy(ags_scene* sc) {
  if (!sc) return;
  DeviceGuard g(sc->ctx->device);
  destroy_instanced(sc);
  cudaFree(sc->d.world_verts);
  cudaFree(sc->d.tri_vidx);
  cudaFree(sc->d.nodes);
  cudaFree(sc->d.tris);
  cudaFree(sc->d.env_root);
  cudaFree(sc->d.leaf_tri);
  cudaFree(sc->d.leaf_bary);
  cudaFree(sc->d.sub_tri_off);
  cudaFree(sc->d.sub_poses);
  cudaFree(sc->d.nodes_build);
  cudaFree(sc->d.base_verts);
  cudaFree(sc->d.sub_vert_off);
  delete sc;
}

int32_t ags_scene_n_envs(const ags_scene* sc) { return sc ? sc->n_envs : -1; }

ags_status ags_context_device(const ags_context* ctx, char* name, int32_t name_len, int32_t* sm_count,
                              int32_t* compute_capability) {
  AGS_API_BEGIN
  if (!ctx) return invalid("ctx is NULL");
  cudaDeviceProp prop{};
  cudaError_t e = cudaGetDeviceProperties(&prop, ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (name && name_len > 0) {
    std::strncpy(name, prop.name, (size_t)name_len - 1);
    name[name_len - 1] = '\0';
  }
  if (sm_count) *sm_count = ctx->sm_count;
  if (compute_capability) *compute_capability = prop.major * 10 + prop.minor;
  return AGS_OK;
  AGS_API_END
}

}  // extern "C"

namespace {
struct SceneDeleter {
  void operator()(ags_scene* s) const { ags_scene_destroy(s); }
};
using ScenePtr = std::unique_ptr<ags_scene, SceneDeleter>;

// A fresh scene built from the kept inputs of sc with the given object poses and build flags.
ags_status rebuild_like(ags_context* ctx, const ags_scene* sc, const float* poses, uint32_t flags, ScenePtr& out) {
  ScenePtr fresh(new ags_scene());
  fresh->ctx = ctx;
  fresh->n_envs = sc->n_envs;
  fresh->n_tris = sc->n_tris;
  fresh->n_verts = sc->n_verts;
  fresh->n_subs = sc->n_subs;
  fresh->flags = flags;
  fresh->env_tri_off = sc->env_tri_off;
  fresh->env_vert_off = sc->env_vert_off;
  fresh->env_sub_off = sc->env_sub_off;
  fresh->sub_tri_off = sc->sub_tri_off;
  fresh->sub_seg = sc->sub_seg;
  ags_status st = build_scene(ctx, fresh.get(), sc->h_base.data(), sc->h_vidx.data(), sc->h_sub_vert.data(), poses,
                              sc->h_sub_env.data());
  if (st != AGS_OK) {
    cudaStreamSynchronize(ctx->stream);
    cudaGetLastError();  // a failed allocation must not surface in a later call
    return st;
  }
  out = std::move(fresh);
  return AGS_OK;
}

// sc takes over fresh's device structures (keeping its own handle, host copies and, if asked, its launch
// choices); fresh leaves with sc's old device structures and is destroyed.
void adopt(ags_scene* sc, ScenePtr& fresh, bool keep_launch) {
  fresh->h_base.swap(sc->h_base);
  fresh->h_vidx.swap(sc->h_vidx);
  fresh->h_sub_vert.swap(sc->h_sub_vert);
  fresh->h_sub_env.swap(sc->h_sub_env);
  fresh->h_poses.swap(sc->h_poses);
  fresh->rebuild_ratio = sc->rebuild_ratio;
  if (keep_launch) fresh->launch = sc->launch;
  std::swap(*sc, *fresh);
  fresh.reset();
}
}  // namespace

extern "C" {

ags_status ags_scene_update_poses(ags_context* ctx, ags_scene* sc, const float* poses, int32_t mode) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  if (mode != AGS_UPDATE_REFIT && mode != AGS_UPDATE_REBUILD && mode != AGS_UPDATE_AUTO)
    return invalid("mode must be AGS_UPDATE_REFIT, AGS_UPDATE_REBUILD or AGS_UPDATE_AUTO");
  if (sc->n_subs > 0 && !poses) return invalid("poses is NULL");
  for (int64_t j = 0; j < sc->n_subs; ++j) {
    const float* p = poses + 7 * j;
    for (int k = 0; k < 7; ++k)
      if (!std::isfinite(p[k])) return invalid("non-finite pose");
    double qn = (double)p[3] * p[3] + (double)p[4] * p[4] + (double)p[5] * p[5] + (double)p[6] * p[6];
    if (!(qn > 1e-12)) return invalid("quaternion has zero length");
  }
  DeviceGuard g(ctx->device);
  ags_status st;
  if (sc->objects) {
    st = update_instanced(ctx, sc, poses);  // two levels: rewrite the object table, rebuild the top level
  } else if (mode == AGS_UPDATE_REFIT) {
    if (sc->node_format != kNodeFp32) return invalid("refit needs float32 nodes; use AGS_UPDATE_REBUILD");
    st = refit_scene(ctx, sc, poses);
  } else {
    bool rebuild = true;
    if (mode == AGS_UPDATE_AUTO && sc->node_format == kNodeFp32 && sc->tree_cost_built > 0.0) {
      // refit, and keep the refitted tree unless its cost outgrew the built tree's by rebuild_ratio
      double cost = 0.0;
      if ((st = refit_scene(ctx, sc, poses)) != AGS_OK || (st = tree_cost(ctx, sc, &cost)) != AGS_OK) return st;
      rebuild = cost > sc->rebuild_ratio * sc->tree_cost_built;
    }
    if (rebuild) {
      // a fresh scene from the kept inputs, then swap it in (with its own built cost)
      ScenePtr fresh;
      if ((st = rebuild_like(ctx, sc, poses, sc->flags, fresh)) == AGS_OK) adopt(sc, fresh, true);
    }
  }
  if (st == AGS_OK && sc->n_subs > 0) sc->h_poses.assign(poses, poses + 7 * sc->n_subs);
  return st;
  AGS_API_END
}

int32_t ags_scene_node_bytes(const ags_scene* sc) { return sc ? node_bytes_of(sc->node_format) : -1; }

ags_status ags_scene_tree_cost(ags_context* ctx, const ags_scene* sc, double out[2]) {
  AGS_API_BEGIN
  if (!ctx || !sc || !out) return invalid("ctx, scene or out is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  if (sc->objects || sc->node_format != kNodeFp32) return invalid("tree cost needs a single-level scene with float32 nodes");
  DeviceGuard g(ctx->device);
  double c = 0.0;
  ags_status st = tree_cost(ctx, sc, &c);
  out[0] = c;
  out[1] = sc->tree_cost_built;
  return st;
  AGS_API_END
}

ags_status ags_scene_set_rebuild_ratio(ags_scene* sc, double ratio) {
  AGS_API_BEGIN
  if (!sc) return invalid("scene is NULL");
  if (!(ratio >= 1.0) || !std::isfinite(ratio)) return invalid("rebuild ratio must be a finite number >= 1");
  sc->rebuild_ratio = ratio;
  return AGS_OK;
  AGS_API_END
}

ags_status ags_render(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                      float* depth, int32_t* seg, void* stream) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!poses || !depth || !seg) return invalid("poses/depth/seg pointer is NULL");
  DeviceGuard g(ctx->device);
  TraceArgs a{};
  const ags_launch_config cfg = lookup_config(sc, spec);
  if ((st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, depth, seg, a, cfg)) != AGS_OK) return st;
  return launch(ctx, a, static_cast<cudaStream_t>(stream), false, cfg.blocks_per_sm);
  AGS_API_END
}

ags_status ags_render_channels(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                               float* depth, int32_t* seg, const ags_hit_channels* ch, void* stream) {
  ags_render_options opt{ch, nullptr, nullptr};
  return ags_render_ex(ctx, sc, spec, poses, depth, seg, &opt, stream);
}

ags_status ags_render_ex(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                         float* depth, int32_t* seg, const ags_render_options* opt, void* stream) {
  AGS_API_BEGIN
  const ags_hit_channels* ch = opt ? opt->channels : nullptr;
  const ags_stereo* stereo = opt ? opt->stereo : nullptr;
  const float* table = opt ? opt->ray_table : nullptr;
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  if (table && reinterpret_cast<uintptr_t>(table) % 4 != 0) return invalid("ray table not 4-byte aligned");
  if (sc->objects && (ch || stereo || table))
    return invalid("two-level scenes render without channels, stereo or ray tables");
  ags_status st = check_spec(spec, table != nullptr);
  if (st != AGS_OK) return st;
  if (!poses || !depth || !seg) return invalid("poses/depth/seg pointer is NULL");
  if (ch) {
    const void* ps[4] = {ch->face, ch->bary, ch->normal, ch->point};
    for (const void* p : ps)
      if (reinterpret_cast<uintptr_t>(p) % 4 != 0) return invalid("channel pointer not 4-byte aligned");
  }
  DeviceGuard g(ctx->device);
  TraceArgs a{};
  ags_launch_config cfg = lookup_config(sc, spec);
  cfg.tile_w = 8;
  cfg.rays_per_lane = 1;
  if ((st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, depth, seg, a, cfg)) != AGS_OK) return st;
  a.sensor.dirs = table;
  if (table) a.extra |= 4;
  if (ch) {
    a.out_face = ch->face;
    a.out_bary = ch->bary;
    a.out_normal = ch->normal;
    a.out_point = ch->point;
    a.extra |= 1;
  }
  if (stereo) {
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(stereo->baseline[k])) return invalid("stereo baseline is not finite");
      a.baseline[k] = stereo->baseline[k];
    }
    const float eps = stereo->eps == 0.0f ? 1e-4f : stereo->eps;
    if (!(eps > 0.0f && eps < 1.0f)) return invalid("stereo eps must lie in (0, 1)");
    a.shadow_eps = eps;
    a.extra |= 2;
  }
  return launch(ctx, a, static_cast<cudaStream_t>(stream), false, cfg.blocks_per_sm);
  AGS_API_END
}

ags_status ags_render_envs(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const int32_t* env_ids,
                           int32_t n, const float* poses, float* depth, int32_t* seg, void* stream) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (n < 0) return invalid("n < 0");
  if (n > 0 && (!env_ids || !poses || !depth || !seg)) return invalid("env_ids/poses/depth/seg pointer is NULL");
  DeviceGuard g(ctx->device);
  TraceArgs a{};
  const ags_launch_config cfg = lookup_config(sc, spec);
  if ((st = fill_trace_args(ctx, sc, spec, n, env_ids, poses, depth, seg, a, cfg)) != AGS_OK) return st;
  return launch(ctx, a, static_cast<cudaStream_t>(stream), false, cfg.blocks_per_sm);
  AGS_API_END
}

ags_status ags_stream_status(ags_context* ctx, void* stream) {
  AGS_API_BEGIN
  if (!ctx) return invalid("ctx is NULL");
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int word = 0;
  if ((e = cudaMemcpyAsync(&word, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return cuda_fail(e, "status word");
  if (word & kStatusBadPose) {
    set_error("a sensor pose was not finite or had a zero-length quaternion; its rays are NaN");
    return AGS_ERR_INVALID_ARG;
  }
  if (word != 0) {
    set_error(std::string("device traversal limit hit:") + ((word & kStatusStackOverflow) ? " stack" : "") +
              ((word & kStatusIterationCap) ? " iterations" : "") +
              ((word & kStatusBadIndex) ? " out-of-range index" : ""));
    return AGS_ERR_TRAVERSAL_LIMIT;
  }
  return AGS_OK;
  AGS_API_END
}

}  // extern "C"

namespace {
// The device address of page-locked host memory (cudaHostAlloc / cudaHostRegister), or null.
void* mapped_host(const void* h) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}
}  // namespace

extern "C" {

ags_status ags_render_host(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const float* poses_h,
                           float* depth_h, int32_t* seg_h) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!poses_h || !depth_h || !seg_h) return invalid("poses/depth/seg pointer is NULL");
  DeviceGuard g(ctx->device);
  const int64_t n = sc->n_envs, pix = (int64_t)spec->width * spec->height;
  const size_t pose_b = ((size_t)n * 7 * sizeof(float) + 255) & ~size_t(255);
  const size_t out_b = ((size_t)(n * pix) * sizeof(float) + 255) & ~size_t(255);
  // page-locked outputs: the kernel writes them in place over the host link (no staging, no copy-back)
  float* depth_m = static_cast<float*>(mapped_host(depth_h));
  int32_t* seg_m = static_cast<int32_t*>(mapped_host(seg_h));
  const bool direct = depth_m && seg_m;
  const size_t need = pose_b + (direct ? 0 : 2 * out_b);
  cudaError_t e;
  if (ctx->stage_bytes < need) {
    cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    if ((e = cudaMalloc(&ctx->stage, need)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(staging)");
    ctx->stage_bytes = need;
  }
  char* base = static_cast<char*>(ctx->stage);
  float* d_pose = reinterpret_cast<float*>(base);
  float* d_depth = reinterpret_cast<float*>(base + pose_b);
  int32_t* d_seg = reinterpret_cast<int32_t*>(base + pose_b + out_b);
  cudaStream_t s = ctx->stream;
  if ((e = cudaMemcpyAsync(d_pose, poses_h, (size_t)n * 7 * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(poses)");
  TraceArgs a{};
  const ags_launch_config cfg = lookup_config(sc, spec);
  if (direct) {
    if ((st = fill_trace_args(ctx, sc, spec, (int32_t)n, nullptr, d_pose, depth_m, seg_m, a, cfg)) != AGS_OK) return st;
    if ((st = launch(ctx, a, s, false, cfg.blocks_per_sm)) != AGS_OK) return st;
    return ags_stream_status(ctx, s);
  }
  if ((st = fill_trace_args(ctx, sc, spec, (int32_t)n, nullptr, d_pose, d_depth, d_seg, a, cfg)) != AGS_OK) return st;
  if ((st = launch(ctx, a, s, false, cfg.blocks_per_sm)) != AGS_OK) return st;
  if ((e = cudaMemcpyAsync(depth_h, d_depth, (size_t)(n * pix) * sizeof(float), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(seg_h, d_seg, (size_t)(n * pix) * sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(outputs)");
  return ags_stream_status(ctx, s);
  AGS_API_END
}

ags_status ags_render_count(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                            uint64_t counts_host[3]) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!poses || !counts_host) return invalid("poses/counts pointer is NULL");
  if (sc->objects) return invalid("counting needs a single-level scene");
  DeviceGuard g(ctx->device);
  TraceArgs a{};
  if ((st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, nullptr, nullptr, a, default_config())) !=
      AGS_OK)
    return st;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemsetAsync(ctx->d_counts, 0, 3 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counts)");
  if ((st = launch(ctx, a, s, true)) != AGS_OK) return st;
  unsigned long long c[3];
  if ((e = cudaMemcpyAsync(c, ctx->d_counts, sizeof(c), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(counts)");
  st = ags_stream_status(ctx, s);
  for (int k = 0; k < 3; ++k) counts_host[k] = c[k];
  return st;
  AGS_API_END
}

ags_status ags_scene_get_world_triangles(const ags_scene* sc, int32_t env, float* out, int32_t* out_seg,
                                         int64_t capacity) {
  AGS_API_BEGIN
  if (!sc) return invalid("scene is NULL");
  if (env < 0 || env >= sc->n_envs) return invalid("env out of range");
  int64_t f0 = sc->env_tri_off[env], f1 = sc->env_tri_off[env + 1];
  int64_t v0 = sc->env_vert_off[env], v1 = sc->env_vert_off[env + 1];
  int64_t n = f1 - f0;
  if (capacity < n) return invalid("capacity smaller than the environment's triangle count");
  if (n == 0) return AGS_OK;
  if (!out || !out_seg) return invalid("output pointer is NULL");
  DeviceGuard g(sc->ctx->device);
  std::vector<float4> verts(v1 - v0);
  std::vector<int32_t> idx(3 * n);
  cudaStream_t s = sc->ctx->stream;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(verts.data(), sc->d.world_verts + v0, verts.size() * sizeof(float4), cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(idx.data(), sc->d.tri_vidx + 3 * f0, idx.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "world triangle readback");
  for (int64_t t = 0; t < n; ++t)
    for (int c = 0; c < 3; ++c) {
      const float4& v = verts[idx[3 * t + c] - v0];
      out[9 * t + 3 * c] = v.x;
      out[9 * t + 3 * c + 1] = v.y;
      out[9 * t + 3 * c + 2] = v.z;
    }
  for (int64_t j = sc->env_sub_off[env]; j < sc->env_sub_off[env + 1]; ++j)
    for (int64_t t = sc->sub_tri_off[j]; t < sc->sub_tri_off[j + 1]; ++t) out_seg[t - f0] = sc->sub_seg[j];
  return AGS_OK;
  AGS_API_END
}

ags_status ags_scene_stats(const ags_scene* sc, int32_t env, int64_t* n_tris, int64_t* n_nodes, int64_t* bytes) {
  AGS_API_BEGIN
  if (!sc) return invalid("scene is NULL");
  if (env < -1 || env >= sc->n_envs) return invalid("env out of range");
  int64_t t, nd, refs;
  if (env == -1) {
    t = sc->n_tris;
    nd = sc->n_nodes;
    refs = sc->n_refs;
  } else {
    t = sc->env_tri_off[env + 1] - sc->env_tri_off[env];
    nd = sc->env_nodes[env];
    refs = sc->env_ref_off.empty() ? 0 : sc->env_ref_off[env + 1] - sc->env_ref_off[env];
  }
  if (n_tris) *n_tris = t;
  if (n_nodes) *n_nodes = nd;
  if (bytes) *bytes = nd * (int64_t)node_bytes_of(sc->node_format) + refs * kTriFloat4 * (int64_t)sizeof(float4);
  return AGS_OK;
  AGS_API_END
}

}  // extern "C"

struct ags_graph {
  ags_context* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned int* counter = nullptr;
};

extern "C" {

ags_status ags_render_graph_create(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec,
                                   const float* poses, float* depth, int32_t* seg, ags_graph** out) {
  AGS_API_BEGIN
  if (!out) return invalid("out is NULL");
  *out = nullptr;
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!poses || !depth || !seg) return invalid("poses/depth/seg pointer is NULL");
  DeviceGuard g(ctx->device);
  std::unique_ptr<ags_graph> gr(new ags_graph());
  gr->ctx = ctx;
  cudaError_t e = cudaMalloc(&gr->counter, sizeof(unsigned int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(graph counter)");
  TraceArgs a{};
  const ags_launch_config cfg = lookup_config(sc, spec);
  if ((st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, depth, seg, a, cfg)) != AGS_OK) {
    cudaFree(gr->counter);
    return st;
  }
  a.tile_counter = gr->counter;
  cudaStream_t s = ctx->stream;
  if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
    cudaFree(gr->counter);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  cudaMemsetAsync(gr->counter, 0, sizeof(unsigned int), s);
  const int blocks = cfg.blocks_per_sm > 0 ? ctx->sm_count * cfg.blocks_per_sm : ctx->trace_blocks;
  cudaError_t le = a.total_tiles > 0 ? launch_trace(a, blocks, false, s) : cudaSuccess;
  e = cudaStreamEndCapture(s, &gr->graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (gr->graph) cudaGraphDestroy(gr->graph);
    cudaFree(gr->counter);
    return cuda_fail(le != cudaSuccess ? le : e, "graph capture");
  }
  if ((e = cudaGraphInstantiate(&gr->exec, gr->graph, 0)) != cudaSuccess) {
    cudaGraphDestroy(gr->graph);
    cudaFree(gr->counter);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  *out = gr.release();
  return AGS_OK;
  AGS_API_END
}

ags_status ags_render_graph_launch(ags_graph* gr, void* stream) {
  if (!gr) return invalid("graph is NULL");
  DeviceGuard g(gr->ctx->device);
  cudaError_t e = cudaGraphLaunch(gr->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? AGS_OK : cuda_fail(e, "cudaGraphLaunch");
}

void ags_render_graph_destroy(ags_graph* gr) {
  if (!gr) return;
  DeviceGuard g(gr->ctx->device);
  cudaDeviceSynchronize();
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  cudaFree(gr->counter);
  delete gr;
}

ags_status ags_memcpy_d2h(void* dst, const void* src, int64_t bytes) {
  if (bytes < 0 || (bytes > 0 && (!dst || !src))) return invalid("bad ags_memcpy_d2h arguments");
  if (bytes == 0) return AGS_OK;
  cudaError_t e = cudaMemcpy(dst, src, (size_t)bytes, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? AGS_OK : cuda_fail(e, "cudaMemcpy");
}

ags_status ags_set_launch_config(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec,
                                 const ags_launch_config* config) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!config) {
    sc->launch.erase({spec->type, spec->width, spec->height});
    return AGS_OK;
  }
  if ((st = check_config(ctx, config)) != AGS_OK) return st;
  if (sc->objects && (config->tile_w != 8 || config->rays_per_lane != 1 ||
                      (config->stack_depth != 0 && config->stack_depth != 64)))
    return invalid("two-level scenes render with the 8x4 tile and the full stack");
  sc->launch[{spec->type, spec->width, spec->height}] = *config;
  return AGS_OK;
  AGS_API_END
}

ags_status ags_get_launch_config(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec,
                                 ags_launch_config* config) {
  AGS_API_BEGIN
  if (!ctx || !sc || !config) return invalid("ctx, scene or config is NULL");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  *config = lookup_config(sc, spec);
  return AGS_OK;
  AGS_API_END
}

ags_status ags_autotune(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                        float* depth, int32_t* seg, int32_t repeats, ags_launch_config* best) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!poses || !depth || !seg || !best) return invalid("poses/depth/seg/best pointer is NULL");
  if (repeats < 1 || repeats > 1000) return invalid("repeats must be in [1, 1000]");
  DeviceGuard g(ctx->device);

  const int full = max_blocks_per_sm(ctx);
  const int grids[2] = {0, full > 2 ? full - 2 : 0};
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  ags_launch_config top = default_config();
  top.ms = -1.0f;
  st = AGS_OK;
  for (int gi = 0; gi < 2 && st == AGS_OK; ++gi) {
    if (gi == 1 && grids[1] == 0) break;
    for (int k = 0; k < kTraceShapes && st == AGS_OK; ++k) {
      if (sc->objects && (kTraceShape[k][0] != 8 || kTraceShape[k][1] != 1)) continue;  // two levels: 8x4 only
      ags_launch_config c = {kTraceShape[k][0], kTraceShape[k][1], grids[gi], 0.0f};
      TraceArgs a{};
      if ((st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, depth, seg, a, c)) != AGS_OK) break;
      if ((st = launch(ctx, a, s, false, c.blocks_per_sm)) != AGS_OK) break;
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess) {
        st = cuda_fail(e, "cudaEventRecord");
        break;
      }
      for (int r = 0; r < repeats && st == AGS_OK; ++r) st = launch(ctx, a, s, false, c.blocks_per_sm);
      if (st != AGS_OK) break;
      float ms = 0.0f;
      if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        st = cuda_fail(e, "autotune timing");
        break;
      }
      c.ms = ms / repeats;
      // the default shape is timed first; another replaces the best only when
      // more than 1% faster, so near ties (within run-to-run noise) keep it
      if (top.ms < 0.0f || c.ms < 0.99f * top.ms) top = c;
    }
  }
  // the stack depth: the 8x4 tile with 32 and 16 stack entries (rays that need more are walked again with
  // 64, so results do not change); a candidate whose retry list overflowed is skipped
  for (int sd : {32, 16}) {
    if (st != AGS_OK || sc->objects) break;
    ags_launch_config c = {8, 1, 0, 0.0f, sd};
    TraceArgs a{};
    if ((st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, depth, seg, a, c)) != AGS_OK) break;
    if ((st = launch(ctx, a, s, false, 0)) != AGS_OK) break;
    unsigned int listed = 0;
    if ((e = cudaMemcpyAsync(&listed, ctx->d_retry_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      st = cuda_fail(e, "autotune retry count");
      break;
    }
    if (listed > (unsigned int)ctx->retry_cap) {
      int word = 0;  // clear the overflow this candidate reported
      if ((e = cudaMemcpy(&word, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
          (e = cudaMemset(ctx->d_status, 0, sizeof(int))) != cudaSuccess) {
        st = cuda_fail(e, "autotune status");
        break;
      }
      continue;
    }
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) {
      st = cuda_fail(e, "cudaEventRecord");
      break;
    }
    for (int r = 0; r < repeats && st == AGS_OK; ++r) st = launch(ctx, a, s, false, 0);
    if (st != AGS_OK) break;
    float ms = 0.0f;
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
        (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
      st = cuda_fail(e, "autotune timing");
      break;
    }
    c.ms = ms / repeats;
    if (c.ms < 0.99f * top.ms) top = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != AGS_OK) return st;
  if ((st = ags_stream_status(ctx, s)) != AGS_OK) return st;
  sc->launch[{spec->type, spec->width, spec->height}] = top;
  *best = top;
  return AGS_OK;
  AGS_API_END
}

}  // extern "C"

namespace {
// Mean time of `repeats` renders of every environment (default launch shape), after one warm-up.
ags_status time_render(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                       float* depth, int32_t* seg, int repeats, float* ms) {
  cudaStream_t s = ctx->stream;
  TraceArgs a{};
  const ags_launch_config c = default_config();
  ags_status st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, depth, seg, a, c);
  if (st != AGS_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  st = launch(ctx, a, s, false, 0);
  if (st == AGS_OK && (e = cudaEventRecord(e0, s)) != cudaSuccess) st = cuda_fail(e, "cudaEventRecord");
  for (int r = 0; r < repeats && st == AGS_OK; ++r) st = launch(ctx, a, s, false, 0);
  if (st == AGS_OK && ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                       (e = cudaEventElapsedTime(ms, e0, e1)) != cudaSuccess))
    st = cuda_fail(e, "build tuning timing");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != AGS_OK) return st;
  *ms /= repeats;
  return ags_stream_status(ctx, s);
}
}  // namespace

extern "C" {

ags_status ags_render_bruteforce(ags_context* ctx, const ags_scene* sc, const ags_sensor_spec* spec,
                                 const float* poses, float* depth, int32_t* seg, void* stream) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  if (sc->objects) return invalid("brute force needs a single-level scene");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!poses || !depth || !seg) return invalid("poses/depth/seg pointer is NULL");
  DeviceGuard g(ctx->device);
  TraceArgs a{};
  if ((st = fill_trace_args(ctx, sc, spec, sc->n_envs, nullptr, poses, depth, seg, a, default_config())) != AGS_OK)
    return st;
  const int32_t E = sc->n_envs, R = (int32_t)sc->n_refs;
  if ((int64_t)sc->env_ref_off.size() != E + 1 || (int64_t)sc->env_tri_off.size() != E + 1)
    return invalid("scene offsets are missing");
  std::vector<int32_t> off(2 * ((size_t)E + 1));
  for (int32_t e = 0; e <= E; ++e) {
    off[e] = (int32_t)sc->env_ref_off[e];
    off[E + 1 + e] = (int32_t)sc->env_tri_off[e];
  }
  DevBufs tmp;
  int32_t* d_off = nullptr;
  char* d_temp = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = tmp.alloc(&d_off, off.size())) != cudaSuccess || (e = tmp.alloc(&d_temp, brute_temp_bytes(R))) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = launch_brute(a, d_off, d_off + E + 1, sc->d.leaf_tri, E, R, d_temp, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "brute-force render");
  return AGS_OK;
  AGS_API_END
}

ags_status ags_test_sort_pairs(ags_context* ctx, uint64_t* keys, uint32_t* vals, int64_t n, int32_t end_bit) {
  AGS_API_BEGIN
  if (!ctx) return invalid("ctx is NULL");
  if (n < 0 || n >= (1ll << 31)) return invalid("n must be in [0, 2^31)");
  if (n > 0 && (!keys || !vals)) return invalid("keys or vals is NULL");
  if (end_bit < 1 || end_bit > 64) return invalid("end_bit must be in [1, 64]");
  DeviceGuard g(ctx->device);
  DevBufs tmp;
  uint64_t* k2 = nullptr;
  uint32_t* v2 = nullptr;
  char* t = nullptr;
  cudaError_t e;
  if ((e = tmp.alloc(&k2, (size_t)n)) != cudaSuccess || (e = tmp.alloc(&v2, (size_t)n)) != cudaSuccess ||
      (e = tmp.alloc(&t, sort_temp_bytes(n))) != cudaSuccess)
    return cuda_fail(e, "sort scratch");
  if ((e = sort_pairs(keys, vals, k2, v2, n, end_bit, t, ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return cuda_fail(e, "sort_pairs");
  return AGS_OK;
  AGS_API_END
}

ags_status ags_test_exclusive_scan(ags_context* ctx, int32_t* data, int64_t n, int32_t* total_host) {
  AGS_API_BEGIN
  if (!ctx || !total_host) return invalid("ctx or total is NULL");
  if (n < 0 || n >= (1ll << 31)) return invalid("n must be in [0, 2^31)");
  if (n > 0 && !data) return invalid("data is NULL");
  DeviceGuard g(ctx->device);
  DevBufs tmp;
  int32_t* total = nullptr;
  char* t = nullptr;
  cudaError_t e;
  if ((e = tmp.alloc(&total, 1)) != cudaSuccess || (e = tmp.alloc(&t, scan_temp_bytes(n))) != cudaSuccess)
    return cuda_fail(e, "scan scratch");
  if ((e = exclusive_scan(data, n, total, t, ctx->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(total_host, total, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return cuda_fail(e, "exclusive_scan");
  return AGS_OK;
  AGS_API_END
}

ags_status ags_autotune_build_flags(ags_context* ctx, ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                                    float* depth, int32_t* seg, const uint32_t* flags, int32_t n_flags, int32_t repeats,
                                    uint32_t* best_flags) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->ctx != ctx) return invalid("scene belongs to another context");
  if (sc->objects) return invalid("build tuning needs a single-level scene");
  ags_status st = check_spec(spec, false);
  if (st != AGS_OK) return st;
  if (!poses || !depth || !seg || !best_flags || (n_flags > 0 && !flags)) return invalid("NULL pointer argument");
  if (n_flags < 0 || n_flags > 64) return invalid("n_flags must be in [0, 64]");
  if (repeats < 1 || repeats > 1000) return invalid("repeats must be in [1, 1000]");
  for (int32_t k = 0; k < n_flags; ++k) {
    const uint32_t f = flags[k];
    if ((f & 0xFFu) > AGS_BVH_Q8) return invalid("unsupported BVH node format in a candidate");
    if ((f & ~(0xFFFFFu | AGS_BUILD_LBVH | AGS_BUILD_GREEDY_COLLAPSE | AGS_CLUSTER_RADIUS(128))) != 0)
      return invalid("unknown bits in a candidate (two-level scenes are not tuned)");
    if (((f >> 8) & 0xFu) > (uint32_t)kMaxLeafTris) return invalid("leaf size must be 1..4");
  }
  if (sc->n_subs > 0 && sc->h_poses.size() != 7 * (size_t)sc->n_subs) return invalid("scene has no kept poses");
  DeviceGuard g(ctx->device);
  float best_ms = 0.0f;
  if ((st = time_render(ctx, sc, spec, poses, depth, seg, repeats, &best_ms)) != AGS_OK) return st;
  uint32_t best = sc->flags;
  const float* h_poses = sc->n_subs > 0 ? sc->h_poses.data() : nullptr;
  for (int32_t k = 0; k < n_flags; ++k) {
    if (flags[k] == best) continue;
    ScenePtr cand;
    st = rebuild_like(ctx, sc, h_poses, flags[k], cand);
    if (st == AGS_ERR_OUT_OF_MEMORY) continue;  // this setting does not fit beside the scene: skip it
    if (st != AGS_OK) return st;
    float ms = 0.0f;
    if ((st = time_render(ctx, cand.get(), spec, poses, depth, seg, repeats, &ms)) != AGS_OK) return st;
    if (ms < best_ms) {  // keep the faster BVH at once, so at most two are held during tuning
      best_ms = ms;
      best = flags[k];
      adopt(sc, cand, false);
    }
  }
  *best_flags = best;
  return AGS_OK;
  AGS_API_END
}

ags_status ags_autotune_build(ags_context* ctx, ags_scene* sc, const ags_sensor_spec* spec, const float* poses,
                              float* depth, int32_t* seg, const uint32_t* cells, int32_t n_cells, int32_t repeats,
                              uint32_t* best_cells) {
  AGS_API_BEGIN
  if (!ctx || !sc) return invalid("ctx or scene is NULL");
  if (sc->objects) return invalid("splitting tuning needs a single-level scene");
  if (!best_cells || (n_cells > 0 && !cells)) return invalid("NULL pointer argument");
  if (n_cells < 0 || n_cells > 64) return invalid("n_cells must be in [0, 64]");
  for (int32_t k = 0; k < n_cells; ++k)
    if (cells[k] > 255u) return invalid("split cell counts must be in [0, 255]");
  // the scene's flags with each listed splitting setting
  const uint32_t split_mask = 0xFFu << 12;
  std::vector<uint32_t> cand((size_t)n_cells);
  for (int32_t k = 0; k < n_cells; ++k) cand[k] = (sc->flags & ~split_mask) | (cells[k] << 12);
  uint32_t best = 0;
  ags_status st = ags_autotune_build_flags(ctx, sc, spec, poses, depth, seg, cand.data(), n_cells, repeats, &best);
  if (st != AGS_OK) return st;
  *best_cells = (best >> 12) & 0xFFu;
  return AGS_OK;
  AGS_API_END
}

}  // extern "C"
