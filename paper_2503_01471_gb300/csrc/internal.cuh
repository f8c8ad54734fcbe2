// Internal declarations of the GB300 ray-cast renderer (product code only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ags.h"

namespace ags {

// ----------------------------------------------------------------- wide BVH
// 8-wide node, float32 child boxes in structure-of-arrays order so a thread
// reads a whole node with 13 aligned 16-byte loads. The ni inner children sit
// in slots 0..ni-1 and are nodes child_base + slot; leaf children follow, and
// the triangles of all leaf children are contiguous from tri_base; empty
// slots come last. meta[k] (byte k of meta_lo/meta_hi): inner slot 0x80 | ni;
// leaf slot (offset << 2) | (count - 1), its triangles starting at tri_base +
// offset; empty slot 0xFF. So ni = meta byte 0 & 0xF when its top bit is set,
// else 0.
struct __align__(16) WideNode {
  int32_t child_base;
  int32_t tri_base;
  uint32_t meta_lo;
  uint32_t meta_hi;
  float lox[8], hix[8], loy[8], hiy[8], loz[8], hiz[8];
};
static_assert(sizeof(WideNode) == 208, "WideNode layout");

// node formats of the traversal (ags_scene_build flags, bits 0-7)
constexpr int kNodeFp32 = 0;  // WideNode, 208 B
constexpr int kNodeFp16 = 1;  // 128 B: child bounds as float16 offsets from the node's origin
constexpr int kNodeQ8 = 2;    // 80 B: child bounds as 8-bit steps of a power-of-two scale per axis
inline int node_bytes_of(int fmt) { return fmt == kNodeFp16 ? 128 : (fmt == kNodeQ8 ? 80 : 208); }

constexpr int kMaxLeafTris = 4;      // largest wide-BVH leaf (2-bit count field)
// weights of the surface-area cost model of the wide tree (ploc.cu's collapse and tree_cost): a wide
// node visit against a triangle test, about the ratio of their instructions
#ifndef AGS_SAH_TRI_COST
#define AGS_SAH_TRI_COST 0.3f
#endif
constexpr float kSahNodeCost = 1.0f, kSahTriCost = AGS_SAH_TRI_COST;
constexpr int kDefaultLeafTris = 2;  // default leaf size (fewest instructions per ray on room scenes)
constexpr uint8_t kMetaEmpty = 0xFF;
constexpr float kEmptyBoxCoord = 1e30f;  // empty slots hold a far-away point box

// Packed triangle: three float4, xyz = world vertex; w of the first holds the
// segment ID bits, w of the second the triangle's index within its
// environment (tie-break key), w of the third is unused.
constexpr int kTriFloat4 = 3;

// device status word bits
constexpr int kStatusStackOverflow = 1;
constexpr int kStatusIterationCap = 2;
constexpr int kStatusBadIndex = 4;
constexpr int32_t kRetryAlloc = 1 << 20;  // retry-list entries each context holds (8 MiB)
constexpr int kStatusBadPose = 8;

// ----------------------------------------------------------------- scene
struct SceneDevice {
  float4* world_verts = nullptr;   // [V] xyz world, w 0
  int32_t* tri_vidx = nullptr;     // [3F] global vertex indices (input order)
  void* nodes = nullptr;           // [n_nodes] in the scene's node format
  float4* tris = nullptr;          // [3R] packed, one per BVH reference, leaf order
  int32_t* env_root = nullptr;     // [E] root node index, -1 if empty
  int32_t* leaf_tri = nullptr;     // [R] input triangle of each leaf-order copy
  uint2* leaf_bary = nullptr;      // [R] barycentric range of each copy's piece (float32 nodes only)
  float* base_verts = nullptr;     // [3V] object-frame vertices (for pose updates)
  int32_t* sub_vert_off = nullptr; // [J+1]
  int32_t* sub_tri_off = nullptr;  // [J+1] (refit: sub-mesh of a triangle)
  float* sub_poses = nullptr;      // [J][7] poses the BVH was built with
  WideNode* nodes_build = nullptr; // refit: copy of the nodes as built, taken at the first refit
};

struct Box {
  float lox, loy, loz, hix, hiy, hiz;
};

// One object of a two-level scene: the rotation that takes world vectors to
// the object's frame, its position, the root of its own BVH and its first
// triangle within its environment.
struct InstanceDev {
  float rt[9];          // R(q)^T, row-major
  float p[3];
  int32_t root;         // wide node in the object-level pool, -1 for an empty object
  int32_t tri_base;     // environment-local index of the object's first triangle
  int32_t pad[2];
};
static_assert(sizeof(InstanceDev) == 64, "InstanceDev layout");

// One entry of a two-level scene's top level: a part of object j's BVH that
// the top level holds under its own world box (the object's root, or one
// child of the root when the root is opened into the top level). node >= 0:
// the walk starts at that node of the object-level pool; node < 0: the part
// is a leaf, triangles leaf_start .. leaf_start + leaf_cnt - 1 of the pool.
struct ObjPart {
  double box[6];  // object-frame bounds
  int32_t node, leaf_start, leaf_cnt;
};

}  // namespace ags

struct ags_context {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;       // internal stream for builds and host renders
  int* d_status = nullptr;             // device status word
  unsigned long long* d_counts = nullptr;  // [3] counters for ags_render_count
  std::map<cudaStream_t, unsigned int*> tile_counters;
  int trace_blocks = 0;                // persistent grid size
  int32_t max_node_visits = 1 << 20;   // per-ray traversal cap
  // short-stack renders: rays whose stack ran out, walked again with the full stack
  int64_t* d_retry_list = nullptr;
  unsigned int* d_retry_count = nullptr;
  int32_t retry_cap = 0;               // in use (<= the allocated kRetryAlloc)
  int trace_count_blocks = 0;
  // staging for ags_render_host
  void* stage = nullptr;
  size_t stage_bytes = 0;
};

struct LaunchKey {
  int32_t type, width, height;
  bool operator<(const LaunchKey& o) const {
    return type != o.type ? type < o.type : (width != o.width ? width < o.width : height < o.height);
  }
};

struct ags_scene {
  ags_context* ctx = nullptr;
  int32_t n_envs = 0;
  int64_t n_tris = 0, n_verts = 0, n_subs = 0, n_nodes = 0;
  int64_t n_refs = 0;                  // BVH references (triangles, some split into several)
  int node_format = 0;                 // kNodeFp32 / kNodeFp16 / kNodeQ8
  uint32_t flags = 0;
  ags::SceneDevice d;
  std::vector<int64_t> env_tri_off;    // [E+1]
  std::vector<int64_t> env_vert_off;   // [E+1]
  std::vector<int64_t> env_sub_off;    // [E+1]
  std::vector<int64_t> sub_tri_off;    // [J+1]
  std::vector<int32_t> sub_seg;        // [J]
  std::vector<int64_t> env_nodes;      // [E]
  std::vector<int64_t> env_ref_off;    // [E+1]
  std::vector<int64_t> level_off;      // wide-node index where each collapse level starts (+ end)
  // host copies of the inputs, for ags_scene_update_poses(..., AGS_UPDATE_REBUILD)
  std::vector<float> h_base;
  std::vector<int32_t> h_vidx, h_sub_vert, h_sub_env;
  std::vector<float> h_poses;  // the current object poses [J][7] (rebuilds start from these)
  mutable std::map<LaunchKey, ags_launch_config> launch;  // tuned or set launch shapes per sensor shape
  // two-level scenes (AGS_BUILD_INSTANCED): a BVH per object in its own frame (`objects`, one
  // environment per object) and per environment a BVH over its objects' world boxes (`top`)
  ags_scene* objects = nullptr;
  ags_scene* top = nullptr;
  ags::InstanceDev* d_inst = nullptr;  // [J]
  int32_t* d_env_sub = nullptr;        // [E+1]
  std::vector<double> h_obj_box;       // [J][6] object-frame bounds of each object's vertices
  std::vector<ags::ObjPart> h_parts;   // the top level's entries of every object, object-major
  std::vector<int64_t> h_part_off;     // [J+1]
  int4* d_parts = nullptr;             // top level of a two-level scene: per leaf reference {object, node,
                                       // leaf start, leaf count}, in leaf order
  // AGS_UPDATE_AUTO: surface-area cost of the float32 tree as built (tree_cost; -1 when not measured)
  // and the multiple of it above which a refitted tree is rebuilt instead
  double tree_cost_built = -1.0;
  double rebuild_ratio = 1.25;
};

namespace ags {

void set_error(const std::string& msg);
ags_status cuda_fail(cudaError_t e, const char* what);

// radix_sort.cu: stable LSD sort of (key, value) pairs over bits [0, end_bit).
// keys/vals hold the input and receive the output; alt_* are scratch of the
// same size. temp must hold sort_temp_bytes(n) bytes.
size_t sort_temp_bytes(int64_t n);
cudaError_t sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* alt_keys, uint32_t* alt_vals,
                       int64_t n, int end_bit, void* temp, cudaStream_t s);
// exclusive scan of n int32 values in place; returns the total in *total_dev (device int)
size_t scan_temp_bytes(int64_t n);
cudaError_t exclusive_scan(int32_t* data, int64_t n, int32_t* total_dev, void* temp, cudaStream_t s);

// An NVTX range over a scope (shown by profilers that record NVTX; free when none is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// device scratch freed when the holder goes out of scope
struct DevBufs {
  std::vector<void*> ptrs;
  DevBufs() = default;
  DevBufs(const DevBufs&) = delete;
  DevBufs& operator=(const DevBufs&) = delete;
  ~DevBufs() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (count > 1 ? count : 1) * sizeof(T));
    if (e == cudaSuccess) {
      ptrs.push_back(q);
      *p = static_cast<T*>(q);
    }
    return e;
  }
};

#define AGS_CHECK(call)                                 \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

// ploc.cu: binary BVH by locally-ordered clustering over the R references
// sorted environment-major by Morton code (keys, vals). Writes inner nodes
// 0..n_inner-1 (left/right: inner id, or ~position of a leaf), their boxes
// and depth-first position ranges [first, last]; reorders vals and writes
// leaf_box in that depth-first order; roots[e] = root of environment e
// (inner id, ~position for a single reference, -1 when empty). With a
// non-null `choice` [R], also the surface-area-optimal wide-node slots of
// every inner node for leaves of up to leaf_max references (see
// collapse_choice in ploc.cu).
ags_status build_ploc(const uint64_t* keys, uint32_t* vals, int32_t R, int key_shift, const int32_t* env_ref_off,
                      int32_t E, const Box* ref_box, Box* leaf_box, int32_t* left, int32_t* right, int32_t* first,
                      int32_t* last, Box* inner_box, std::vector<int32_t>& roots, cudaStream_t s,
                      uint32_t* choice = nullptr, int leaf_max = 2, int radius = 16);

// build.cu: world vertices v' = R(q) v + p of every sub-mesh (float-float, as the scene build)
ags_status transform_vertices(const float* base_dev, int32_t V, const int32_t* sub_vert_off_dev, int32_t J,
                              const float* poses_dev, float4* world_dev, cudaStream_t s);

// instanced.cu: two-level scenes. build_instanced fills sc (its sizes and offsets already set) from the
// host inputs; update_instanced moves the objects; destroy_instanced frees what the two levels hold.
ags_status build_instanced(ags_context* ctx, ags_scene* sc, const float* base_verts_h, const int32_t* tri_vidx_h,
                           const int32_t* sub_vert_off_h, const float* poses_h, const int32_t* sub_env_h);
ags_status update_instanced(ags_context* ctx, ags_scene* sc, const float* poses_h);
void destroy_instanced(ags_scene* sc);

// build.cu
ags_status build_scene(ags_context* ctx, ags_scene* sc, const float* base_verts_h,
                       const int32_t* tri_vidx_h, const int32_t* sub_vert_off_h,
                       const float* poses_h, const int32_t* sub_env_h);

ags_status refit_scene(ags_context* ctx, ags_scene* sc, const float* poses_h);
// surface-area cost of a float32 tree under the collapse's model (kSahNodeCost x area of every inner
// child box + kSahTriCost x count x area of every leaf child box, all nodes); synchronous
ags_status tree_cost(ags_context* ctx, const ags_scene* sc, double* cost);

// trace.cu
// Ray pattern of one sensor shape (derived from ags_sensor_spec on the host).
struct SensorParams {
  int32_t W, H;
  int32_t type;
  int32_t near_mode;
  float inv_f;               // camera: 1/f
  float hfov, vmax, dv;      // LiDAR: azimuth span, top elevation, elevation step
  float min_range, max_range;
  int32_t tiles_x;           // warp tiles across a row for the launch shape
  int32_t tiles_per_env;     // warp tiles per environment
  const float* dirs;         // AGS_RAY_TABLE: [H][W][3] sensor-frame directions
};

// One request of a serving batch (slot mode of the render kernel).
struct SlotEntry {
  int32_t env;
  int32_t spec;              // index into the batch's SensorParams table
  int32_t tile_begin;        // first global tile of this slot
  int32_t pad0;
  int64_t out_offset;        // element offset of this slot's [H][W] outputs
  float pose[7];
  float pad1;
};
static_assert(sizeof(SlotEntry) == 56, "SlotEntry layout");

struct TraceArgs {
  const void* nodes;         // node_format layout
  int32_t node_format;
  const float4* tris;
  const int32_t* env_root;
  int32_t n_nodes;           // bounds for the node and triangle indices read
  int32_t n_tris;
  int32_t n_scene_envs;
  const int32_t* env_ids;    // nullable
  const float* poses;        // [n][7]
  float* out_depth;          // [n][H][W] (slot mode: output arena)
  int32_t* out_seg;
  // extra hit channels (channel kernel only; each nullable): face index
  // [n][H][W], barycentrics [n][H][W][2], world normal and sensor-frame
  // point [n][H][W][3]
  int32_t* out_face;
  float* out_bary;
  float* out_normal;
  float* out_point;
  int32_t extra;             // bit 0: hit channels; bit 1: stereo shadow test; bit 2: ray table
  // two-level scenes: nodes / tris / env_root above are the top level over objects
  int32_t instanced;
  const InstanceDev* inst;
  int32_t n_inst;
  const int32_t* env_sub;    // [E+1] first object of each environment
  const void* obj_nodes;     // object-level pool (float32 nodes)
  const float4* obj_tris;
  int32_t obj_n_nodes, obj_n_tris;
  const int4* parts;         // per top-level leaf reference: {object, node, leaf start, leaf count}
  float baseline[3];         // stereo: second sensor's origin in the sensor frame
  float shadow_eps;          // stereo: the shadow segment starts at this fraction
  int32_t n;                 // environments rendered
  SensorParams sensor;       // uniform mode
  const SensorParams* specs; // slot mode: table of sensor shapes
  int32_t n_specs;
  const SlotEntry* slots;    // slot mode when non-null
  int32_t n_slots;
  const int32_t* slot_header;  // slot mode: when non-null, {n_slots, total_tiles} are read here (device)
  int32_t log2_tile_w, tile_h, rays_per_lane;  // a warp's tile: (1 << log2_tile_w) x tile_h pixels
  int32_t stack_depth;       // plain renders: 16 or 32 walk with a short stack (its overflows retried); else 64
  int64_t* retry_list;       // short stack: output index of every ray to walk again with the full stack
  unsigned int* retry_count;
  int32_t retry_cap;
  int64_t total_tiles;
  int32_t max_visits;
  unsigned int* tile_counter;
  int* status;
  unsigned long long* counts;
};
cudaError_t launch_trace(const TraceArgs& a, int blocks, bool count, cudaStream_t s);
cudaError_t launch_trace_extra(const TraceArgs& a, int blocks, cudaStream_t s);  // a.extra != 0
cudaError_t launch_trace_inst(const TraceArgs& a, int blocks, cudaStream_t s);   // a.instanced != 0
// a plain render with a short stack (a.stack_depth 16 or 32, 8x4 tiles) and its retry pass; the caller has
// zeroed *a.retry_count on the stream
cudaError_t launch_trace_short(const TraceArgs& a, int blocks, int retry_blocks, cudaStream_t s);
// compiled launch shapes of the render kernel: {tile width, rays per lane}
constexpr int kTraceShapes = 7;
constexpr int kTraceShape[kTraceShapes][2] = {{8, 1}, {4, 1}, {8, 2}, {16, 2}, {16, 4}, {16, 1}, {32, 1}};
bool trace_shape_supported(int tile_w, int rays_per_lane);
// host: ray pattern of a validated spec for tiles of tile_w x tile_h
SensorParams sensor_params(const ags_sensor_spec* spec, int tile_w, int tile_h);
int trace_blocks_per_sm(bool count);

}  // namespace ags
