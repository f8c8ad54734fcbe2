/*
 * ags.h -- C ABI of the GB300 batched ray-cast sensor renderer.
 *
 * The operation (Aerial Gym Simulator, Kulkarni, Rehberg, Alexis, IEEE RA-L
 * 2025, Sec. III-D.1 "Exteroceptive Sensors"): every environment i holds a
 * base triangle mesh made of n_i sub-meshes, one per object; each sub-mesh j
 * is moved into the world by its own transform T_j (here a position and a
 * unit quaternion); a bounding volume hierarchy is built over the moved mesh;
 * then one ray per pixel (pinhole camera) or per beam (3-D LiDAR) is cast from
 * each sensor and the nearest intersection reports depth (distance of the hit
 * from the image plane, cameras) or range (distance from the sensor to the
 * hit, LiDAR / time-of-flight), plus the segment ID of the object hit.
 *
 * Conventions (readings of points the paper leaves open):
 *   - pose = (px, py, pz, qx, qy, qz, qw), float32; q need not be unit length
 *     (it is normalised); world vertex v' = R(q) v + p.
 *   - sensor body frame: +x forward (optical axis), +y left, +z up. Camera row
 *     0 is the top row, column 0 the left column; rays pass through pixel
 *     centres; focal length f = (W/2) / tan(hfov/2), square pixels.
 *   - LiDAR: row k = channel at elevation vfov_max - k (vfov_max - vfov_min) /
 *     (H - 1) (row 0 = vfov_max; a single channel sits at vfov_max); column j
 *     = azimuth hfov * j / W counter-clockwise from +x.
 *   - two-sided triangles with closed edges (watertight); nearest hit wins;
 *     equal float32 distance goes to the smaller triangle index within the
 *     environment (sub-meshes concatenated in order).
 *   - min/max range apply to the reported value (depth for cameras, range for
 *     LiDAR); a hit at exactly max_range counts. Misses report exactly
 *     max_range and segment -1. Hits nearer than min_range report min_range
 *     (AGS_NEAR_CLAMP, segment kept) or max_range and -1 (AGS_NEAR_INVALID).
 *
 * Memory: device pointers are CUDA device addresses on the context's device;
 * host pointers are ordinary (pageable or pinned) host memory. Inputs stay
 * owned by the caller. Scenes are owned by the library until
 * ags_scene_destroy. Output buffers are owned by the caller.
 *
 * Errors: every call returns an ags_status and never aborts the process.
 * ags_last_error() returns a thread-local message for the last failure.
 * Kernels never trap: limits hit on the device (traversal stack or iteration
 * cap) set a device status word, returned by ags_stream_status.
 * Thread safety: one context per host thread, or external locking.
 */
#ifndef AGS_H
#define AGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AGS_OK = 0,
  AGS_ERR_INVALID_ARG = 1,    /* bad pointer, size, index, pose or spec */
  AGS_ERR_OUT_OF_MEMORY = 2,  /* device or host allocation failed */
  AGS_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  AGS_ERR_TRAVERSAL_LIMIT = 4,/* a ray hit the stack or iteration limit, or met an out-of-range
                                 index; that ray's output is NaN */
  AGS_ERR_NOT_READY = 5,
  AGS_ERR_BUSY = 6,
  AGS_ERR_CANCELLED = 7       /* a served request cancelled before it was batched */
} ags_status;

typedef struct ags_context ags_context;
typedef struct ags_scene ags_scene;

/* One object (sub-mesh M_j of Sec. III-D.1). Host pointers. */
typedef struct {
  const float* vertices;    /* [n_vertices][3] object frame, metres */
  int32_t n_vertices;
  const int32_t* indices;   /* [n_triangles][3], each in [0, n_vertices) */
  int32_t n_triangles;
  int32_t segment_id;       /* reported for rays that hit this object; >= 0 */
} ags_submesh;

/* One environment: its objects in order. */
typedef struct {
  const ags_submesh* submeshes;
  int32_t n_submeshes;
} ags_env_mesh;

typedef enum { AGS_PINHOLE = 0, AGS_LIDAR = 1, AGS_RAY_TABLE = 2 } ags_sensor_type;
typedef enum { AGS_NEAR_CLAMP = 0, AGS_NEAR_INVALID = 1 } ags_near_mode;

typedef struct {
  int32_t type;          /* ags_sensor_type */
  int32_t width;         /* camera columns / LiDAR azimuth bins, 1..16384 */
  int32_t height;        /* camera rows / LiDAR channels, 1..16384 */
  float hfov_rad;        /* camera horizontal FOV in (0, pi); LiDAR azimuth span in (0, 2 pi] */
  float vfov_min_rad;    /* LiDAR lowest channel elevation (rad), >= -pi/2 */
  float vfov_max_rad;    /* LiDAR highest channel elevation (rad), <= pi/2 */
  float min_range;       /* >= 0 */
  float max_range;       /* > min_range, finite */
  int32_t near_mode;     /* ags_near_mode */
  uint32_t flags;        /* reserved, must be 0 */
} ags_sensor_spec;

/* Build flags: node format of the wide BVH (bits 0-7; every format stores
 * child boxes that contain the exact float32 ones, so results are
 * bit-identical and only the memory per node and the decode work differ);
 * the largest number of
 * triangles in one BVH leaf (bits 8-11: 1..4; 0 selects 2); and the splitting
 * of large triangles into several BVH references (bits 12-19): 0 selects 16
 * cells across an environment's largest extent, 1 turns splitting off, n >= 2
 * uses n cells. A triangle larger than a cell is referenced from up to 8
 * cells per axis (64 in all), each boxed by the triangle clipped to the cell;
 * results are identical with or without splitting. */
#define AGS_BVH_FP32 0u  /* 208-byte nodes, float32 child boxes */
#define AGS_BVH_FP16 1u  /* 128-byte nodes, float16 offsets from the node's origin, rounded outward */
#define AGS_BVH_Q8 2u    /* 80-byte nodes, 8-bit steps of a power-of-two scale per axis, rounded outward */
#define AGS_LEAF_SIZE(n) (((uint32_t)(n) & 0xFu) << 8)
#define AGS_SPLIT_CELLS(n) (((uint32_t)(n) & 0xFFu) << 12)
/* Binary tree under the wide nodes: by default locally-ordered clustering of
 * the Morton-sorted references (lower surface-area cost, slower build); this
 * bit selects the Morton radix tree instead (faster build). Results are
 * identical either way. */
#define AGS_BUILD_LBVH (1u << 20)
/* Wide nodes from the clustered binary tree: by default each node's eight
 * slots are the subtrees of least surface-area cost (a dynamic program over
 * the binary tree); this bit selects the greedy collapse instead (open the
 * largest child until eight slots). The Morton radix tree always uses the
 * greedy collapse. Results are identical either way. */
#define AGS_BUILD_GREEDY_COLLAPSE (1u << 22)
/* Search radius of the clustering (bits 23-24): each round every cluster
 * looks for its partner among r positions on either side in Morton order,
 * r = 16 (the default), 32, 64 or 128. A wider search finds pairs of smaller
 * union boxes, so a tree of lower surface-area cost, at a cost per round
 * proportional to r. Results are identical for every radius. */
#define AGS_CLUSTER_RADIUS(r) \
  ((uint32_t)((r) >= 128 ? 3u : ((r) >= 64 ? 2u : ((r) >= 32 ? 1u : 0u))) << 23)
/* Two-level scene: every object (sub-mesh) gets its own BVH, built once in its
 * own frame without reference splitting (the flags' splitting setting applies
 * to nothing here), and each environment a small BVH over its objects' world
 * boxes (an object whose box has at least a quarter of its environment's box
 * surface, such as a room around the others, enters it as the children of its
 * root, each under its own box); rays are moved into an object's frame to walk
 * its BVH. ags_scene_update_poses
 * then only rebuilds the small top level (either mode). Float32 nodes only; at
 * most 65536 objects; renders through ags_render / ags_render_envs /
 * ags_render_host / step graphs with the 8x4 tile; not with extra channels,
 * stereo, ray tables, counting, splitting tuning or serving (those return
 * AGS_ERR_INVALID_ARG). Results agree with a single-level scene within float32
 * rounding, not bit for bit. */
#define AGS_BUILD_INSTANCED (1u << 21)

/* Launch shape of the persistent render kernel for one (scene, sensor shape):
 * each warp repeatedly takes a tile of tile_w x (32 * rays_per_lane / tile_w)
 * pixels (or beams) of one environment, each lane tracing rays_per_lane rays
 * of it; the grid holds blocks_per_sm blocks per SM (0: as many as fit).
 * stack_depth 16 or 32 (8x4 tile, plain renders) walks each ray with a short
 * traversal stack; a ray that outgrows it is listed and walked again, after
 * the launch, with the full 64-entry stack, so results are the same; the list
 * holds ags_context_set_retry_capacity rays (1048576 by default), beyond which
 * rays report NaN / -1 and AGS_ERR_TRAVERSAL_LIMIT. 0 or 64: the full stack. */
typedef struct {
  int32_t tile_w;         /* with rays_per_lane, one of the compiled shapes: (8,1) 8x4, */
  int32_t rays_per_lane;  /* (4,1) 4x8, (16,1) 16x2, (32,1) 32x1, (8,2) 8x8, (16,2) 16x4, (16,4) 16x8 */
  int32_t blocks_per_sm;  /* 0, or 1 .. the kernel's occupancy limit */
  float ms;               /* ags_autotune: measured time of one render; else 0 */
  int32_t stack_depth;    /* 0 or 64 (full stack), 32 or 16 (short stack with retries) */
} ags_launch_config;

/* Create a context on CUDA device `device`. */
ags_status ags_context_create(int device, ags_context** out);
void ags_context_destroy(ags_context* ctx);

/* The context's device: its name (NUL-terminated, truncated to name_len
 * bytes), SM count and compute capability (major * 10 + minor). Any output
 * pointer may be NULL. */
ags_status ags_context_device(const ags_context* ctx, char* name, int32_t name_len, int32_t* sm_count,
                              int32_t* compute_capability);

/*
 * ags_scene_build -- Sec. III-D.1: transform every sub-mesh by its pose and
 * build one BVH over each environment's meshes M_{i,t}. envs[n_envs]
 * describe the meshes (host memory);
 * obstacle_poses is host float32 [sum_i n_submeshes(i)][7] in environment
 * order, then sub-mesh order. The call validates every input before any
 * device work (indices in range, finite vertices and poses, non-zero
 * quaternions, segment IDs >= 0), copies everything to the device, runs the
 * build kernels on an internal stream and returns once the scene is
 * resident. Limits: 1 <= n_envs <= 65536; total triangles < 2^31 - 1.
 * Environments may be empty (every ray misses).
 */
ags_status ags_scene_build(ags_context* ctx, const ags_env_mesh* envs, int32_t n_envs,
                           const float* obstacle_poses, uint32_t build_flags, ags_scene** out);
void ags_scene_destroy(ags_scene* scene);

/*
 * ags_scene_update_poses -- move every object of a resident scene to new
 * poses (host float32 [sum n_submeshes][7], the order of ags_scene_build):
 * Sec. III-D.1 keeps M_{i,t} current from the transforms T_{j,t} as the
 * simulation runs, there by rebuilding the BVH. AGS_UPDATE_REFIT transforms the
 * vertices, rewrites the packed triangles and refits the node boxes bottom-up
 * in the existing topology (float32 nodes only; fast, but the tree degrades
 * as objects move far); AGS_UPDATE_REBUILD builds the whole scene again with
 * the new poses. Both give exactly the images a freshly built scene gives.
 * Synchronous; the scene must not be in use on any stream meanwhile.
 */
#define AGS_UPDATE_REFIT 0
#define AGS_UPDATE_REBUILD 1
/* AGS_UPDATE_AUTO refits, then rebuilds when the refitted tree's surface-area
 * cost (ags_scene_tree_cost) exceeds the tree's cost as built (or last
 * rebuilt) by more than the scene's rebuild ratio (1.25 unless set); scenes
 * with compressed nodes are rebuilt, two-level scenes update as in the other
 * modes. */
#define AGS_UPDATE_AUTO 2
ags_status ags_scene_update_poses(ags_context* ctx, ags_scene* scene, const float* obstacle_poses, int32_t mode);

/*
 * ags_scene_tree_cost -- the surface-area cost of a single-level scene's
 * float32 BVH under the model its collapse minimises: summed over every wide
 * node, the area (dx dy + dy dz + dz dx) of each inner child box plus 0.3 x
 * triangles x area of each leaf child box. out[0] = now, out[1] = as built or
 * last rebuilt (-1 when not measured). Synchronous. The paper has no
 * counterpart; it tracks how far refits have degraded the tree.
 */
ags_status ags_scene_tree_cost(ags_context* ctx, const ags_scene* scene, double out[2]);
/* The multiple of the built cost above which AGS_UPDATE_AUTO rebuilds (>= 1). */
ags_status ags_scene_set_rebuild_ratio(ags_scene* scene, double ratio);

/*
 * ags_render -- Sec. III-D.1: cast one ray per pixel / beam of `spec` from
 * each environment's sensor pose and report the nearest hit.
 * sensor_poses_dev: device float32 [n_envs][7]. out_depth_dev: device float32
 * [n_envs][height][width] (depth for cameras, range for LiDAR), row-major.
 * out_seg_dev: device int32, same shape. cuda_stream: a cudaStream_t (NULL =
 * legacy default stream). Asynchronous: returns after enqueueing; the outputs
 * are ready when the stream reaches that point. Host-side argument errors are
 * returned immediately with nothing enqueued.
 */
ags_status ags_render(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                      const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                      void* cuda_stream);

/*
 * Extra hit channels (Sec. III-D.1: face indices with barycentric
 * coordinates, surface normals, point clouds). Device buffers owned by the
 * caller, one entry per ray in the layout of the depth output; each pointer
 * may be NULL (that channel is not written); 4-byte aligned.
 *   face    int32 [n_envs][H][W]: env-local index of the triangle hit
 *           (sub-meshes concatenated in build order), -1 on a miss or on a
 *           near hit reported as invalid;
 *   bary    float [n_envs][H][W][2]: (u, v), the weights of that triangle's
 *           second and third vertex at the hit (hit = (1-u-v) v0 + u v1 + v v2);
 *           0 where face is -1;
 *   normal  float [n_envs][H][W][3]: unit geometric normal (v1-v0) x (v2-v0)
 *           in the world frame, turned to face the sensor; 0 where face is -1;
 *   point   float [n_envs][H][W][3]: the hit in the sensor frame, the reported
 *           value times the sensor-frame direction with unit reported
 *           component (camera: depth * (1, a, b), so x = depth; LiDAR:
 *           range * unit direction); misses sit at max_range along the ray.
 * A ray that hits the traversal limits reports NaN weights, normal and point.
 */
typedef struct {
  int32_t* face;
  float* bary;
  float* normal;
  float* point;
} ags_hit_channels;

/*
 * ags_render_channels -- ags_render (bit-identical depth/range and segment
 * IDs) that also writes the extra hit channels listed in `channels` (NULL:
 * none). Uses the 8x4 warp tile whatever launch shape is configured. Errors
 * as ags_render; a misaligned channel pointer -> AGS_ERR_INVALID_ARG.
 */
ags_status ags_render_channels(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                               const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                               const ags_hit_channels* channels, void* cuda_stream);

/*
 * Stereo shadows (Sec. III-D.1: rays projected back from the points of
 * intersection towards the second sensor; pixels whose ray meets the
 * environment are invalid). The second sensor sits at baseline (metres, in
 * the sensor frame: +x forward, +y left, +z up) from the rendered one. A hit
 * P is shadowed when a triangle meets the segment P + s (o2 - P) for s in
 * [eps, 1]; eps (0 -> 1e-4) keeps the surface at P itself out. A shadowed
 * pixel is reported as invalid: max_range, segment -1, face -1.
 */
typedef struct {
  float baseline[3];
  float eps;
} ags_stereo;

/*
 * Options of ags_render_ex; every member may be NULL.
 *   channels   extra hit channels to write;
 *   stereo     stereo shadow invalidation towards a second sensor;
 *   ray_table  device float [height][width][3], the sensor-frame direction
 *              of each pixel of an AGS_RAY_TABLE sensor (a user projection
 *              model, Sec. III-D.1: e.g. a dome LiDAR or a fisheye). The
 *              reported value is the distance along each row in units of its
 *              length: (1, a, b) rows give depth, unit rows give range. Such a
 *              sensor ignores hfov and the elevations; a zero or non-finite
 *              row reports NaN and sets the status as a bad pose does. The
 *              table stays owned by the caller and must outlive the render.
 */
typedef struct {
  const ags_hit_channels* channels;
  const ags_stereo* stereo;
  const float* ray_table;
} ags_render_options;

/*
 * ags_render_ex -- ags_render with the options above (NULL: none). Depth and
 * segment IDs are bit-identical to ags_render where no pixel is shadowed.
 * Uses the 8x4 warp tile. Errors as ags_render; a misaligned channel pointer,
 * a non-finite baseline, eps outside (0, 1), or an AGS_RAY_TABLE sensor
 * without a table (or a table for another sensor type) -> AGS_ERR_INVALID_ARG.
 */
ags_status ags_render_ex(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                         const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                         const ags_render_options* options, void* cuda_stream);

/*
 * ags_render_envs -- as ags_render for the n environments listed in
 * env_ids_dev (device int32 [n], each in [0, n_envs)); sensor_poses_dev is
 * [n][7] and the outputs are [n][height][width], in list order.
 */
ags_status ags_render_envs(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                           const int32_t* env_ids_dev, int32_t n, const float* sensor_poses_dev,
                           float* out_depth_dev, int32_t* out_seg_dev, void* cuda_stream);

/*
 * ags_render_host -- ags_render with HOST buffers: copies sensor_poses_host
 * [n_envs][7] to the device, renders into context-owned device buffers and
 * copies depth/range and segment IDs back into out_depth_host and
 * out_seg_host ([n_envs][height][width]). Synchronous; returns the device
 * status of this render as ags_stream_status would. When both output buffers
 * are page-locked (cudaHostAlloc, cudaHostRegister, torch pin_memory), the
 * render kernel writes them in place through their mapped device addresses
 * (over the host link, no staging buffer and no copy-back); otherwise the
 * outputs are rendered into context-owned device memory and copied back.
 */
ags_status ags_render_host(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                           const float* sensor_poses_host, float* out_depth_host,
                           int32_t* out_seg_host);

/*
 * ags_render_count -- the traversal of ags_render instrumented to count, over
 * all rays, the wide BVH nodes visited and triangles tested (no outputs are
 * written). counts_host receives {rays, nodes visited, triangles tested}.
 * Synchronous. Used to state the algorithmic bytes per ray.
 */
ags_status ags_render_count(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                            const float* sensor_poses_dev, uint64_t counts_host[3]);

/*
 * ags_render_bruteforce -- a test and debugging aid (no counterpart in the
 * paper): the render of ags_render (same outputs, same layouts) with every
 * ray tested against every BVH reference of its environment, no tree, using
 * the render kernel's own ray set-up and triangle test. The BVH walk culls
 * conservatively and breaks ties the same way, so ags_render must match it
 * bit for bit. Cost grows with rays x triangles: meant for checks at reduced
 * resolution. Single-level scenes; camera and LiDAR sensors. Synchronises
 * `cuda_stream`.
 */
ags_status ags_render_bruteforce(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                                 const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                                 void* cuda_stream);

/*
 * Test hooks of two building blocks of ags_scene_build (no counterpart in the
 * paper): the stable LSD radix sort of (uint64 key, uint32 value) pairs on
 * key bits [0, end_bit) (1 <= end_bit <= 64), in place on device buffers, and
 * the exclusive scan of int32 values in place on a device buffer, with the
 * total written to *total_host. Both synchronise the context's stream.
 */
ags_status ags_test_sort_pairs(ags_context* ctx, uint64_t* keys_dev, uint32_t* vals_dev, int64_t n,
                               int32_t end_bit);
ags_status ags_test_exclusive_scan(ags_context* ctx, int32_t* data_dev, int64_t n, int32_t* total_host);

/*
 * ags_scene_validate -- structural checks of the scene's BVH, a test and
 * debugging aid (the paper has no counterpart), run on the host from the
 * device data the render kernel reads: every wide node and every reference
 * reached exactly once from its environment's root, every index in range,
 * each packed triangle copy equal to its source triangle (vertices, segment
 * ID, environment-local index), and every point of a 28-point barycentric
 * grid on every triangle inside all the boxes on the path to one of its
 * references, with boxes decoded from the scene's node format (so a ray that
 * meets a triangle reaches a leaf holding it). Two-level scenes are checked
 * level by level. counts[0] = wide nodes, [1] = points checked, [2] =
 * violations (the first few are described by ags_last_error), [3] = deepest
 * path in nodes. Synchronous; copies the scene to host memory.
 */
ags_status ags_scene_validate(const ags_scene* scene, int64_t counts[4]);

/*
 * ags_autotune_build -- build-time tuning of the reference splitting (the
 * AGS_SPLIT_CELLS setting, 0 = the default 16 cells, 1 = off): the scene is
 * rebuilt, from its kept inputs and current object poses, with each listed
 * setting; `repeats` renders of `spec` (default launch shape, after one
 * warm-up, into the caller's buffers) are timed per setting, and the fastest
 * BVH is kept in `scene` (same handle; results are identical for every
 * setting). *best_cells receives the kept setting. Settings that run out of
 * device memory are skipped. Launch-shape choices of the scene are cleared
 * when its BVH changes (run ags_autotune afterwards). Synchronous. Rebuilds
 * invalidate captured graphs (as AGS_UPDATE_REBUILD does).
 */
ags_status ags_autotune_build(ags_context* ctx, ags_scene* scene, const ags_sensor_spec* spec,
                              const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                              const uint32_t* split_cells, int32_t n_cells, int32_t repeats, uint32_t* best_cells);

/*
 * ags_autotune_build_flags -- the same tuning over whole build settings: each
 * of the n_flags candidates (at most 64) is a build_flags word as for
 * ags_scene_build (node format, leaf size, splitting, clustering radius,
 * builder bits; not AGS_BUILD_INSTANCED), built and timed as above; the
 * fastest BVH, the scene's own included, is kept and *best_flags receives its
 * flags. A candidate with unknown bits is refused (AGS_ERR_INVALID_ARG)
 * before anything is built. ags_autotune_build is this call over the scene's
 * flags with each listed splitting setting.
 */
ags_status ags_autotune_build_flags(ags_context* ctx, ags_scene* scene, const ags_sensor_spec* spec,
                                    const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                                    const uint32_t* flags, int32_t n_flags, int32_t repeats, uint32_t* best_flags);

/*
 * ags_autotune -- time the render of `scene` with `spec` under each compiled
 * launch shape (tiles 8x4, 4x8, 8x8, 16x4, 16x8; full or reduced grid),
 * `repeats` timed renders each after one warm-up, on the context's
 * stream, writing into the caller's buffers (as ags_render). The fastest shape
 * (the default 8x4 tile with the full grid is timed first, and another shape
 * replaces the best so far only when more than 1% faster, so near ties keep
 * the default) is stored with the scene for this sensor shape (type, width, height) and
 * used by every later ags_render / ags_render_envs of that shape; it is also
 * returned in *best. Synchronous. The paper has no counterpart (its renderer
 * is Warp's); the shape does not change any output bit.
 */
ags_status ags_autotune(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                        const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                        int32_t repeats, ags_launch_config* best);

/* Set (or, with config == NULL, clear) the launch shape used for `scene` with
 * sensors of spec's type, width and height. */
ags_status ags_set_launch_config(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                                 const ags_launch_config* config);

/* The launch shape ags_render would use for `scene` and `spec`. */
ags_status ags_get_launch_config(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                                 ags_launch_config* config);

/* ---------------------------------------------------------------- serving
 * A server renders a stream of requests against one resident scene with
 * continuous batching (the paper has no counterpart: there the renderer is
 * called once per simulation step). A worker thread takes waiting requests in
 * arrival order and admits each as soon as a slot of the next batch and room
 * in the device output arena are free (admission by free device memory); it
 * launches the batch (every request with its own environment, sensor shape
 * and pose, in one persistent launch) on one of max_inflight streams, so
 * batches overlap on the GPU while later requests queue. Results stay in the
 * arena -- device memory, for a GPU consumer -- until released. */
typedef struct ags_server ags_server;

typedef struct {
  int32_t max_slots;          /* requests per batch, 1..65536 */
  int32_t max_inflight;       /* batches on the GPU at once (streams), 1..16 */
  int64_t arena_bytes;        /* output arena (8 bytes per ray); 0 = a quarter of free device memory */
  const ags_sensor_spec* specs;  /* sensor shapes requests may use (copied) */
  int32_t n_specs;            /* 1..256 */
  int32_t auto_release;       /* nonzero: free a request's outputs as soon as it completes */
  int32_t use_graph;          /* nonzero: each stream replays one CUDA graph per batch (slot-table copy,
                                 tile-counter reset, render), captured at creation, instead of three calls */
  int32_t pad0;
} ags_server_config;

typedef struct {
  int32_t env;                /* environment of the scene */
  int32_t spec;               /* index into the server's specs */
  float pose[7];              /* sensor pose (px, py, pz, qx, qy, qz, qw) */
  uint64_t tag;               /* caller's value, returned in the completion */
} ags_request;

typedef struct {
  uint64_t request_id;
  uint64_t tag;
  int32_t status;             /* ags_status of the request */
  const float* depth_dev;     /* [H][W] depth / range in the arena (valid until released) */
  const int32_t* seg_dev;     /* [H][W] segment IDs */
  double t_submit, t_start, t_done;  /* host steady-clock seconds: submitted, launched, seen done */
} ags_completion;

/* Create a server on a resident scene (the context's device). Allocates the
 * arena (limited to 90% of the device memory free at creation), per-stream
 * slot tables and a worker thread. */
ags_status ags_server_create(ags_context* ctx, const ags_scene* scene, const ags_server_config* config,
                             ags_server** out);
/* Stop the worker after the requests on the GPU finish; waiting requests are dropped. */
void ags_server_destroy(ags_server* server);
/* Queue a request (validated now; AGS_ERR_BUSY if 2^20 requests wait). Thread-safe. */
ags_status ags_server_submit(ags_server* server, const ags_request* request, uint64_t* request_id);
/* Up to `max` completed requests, oldest first; never blocks. Thread-safe. */
ags_status ags_server_poll(ags_server* server, ags_completion* out, int32_t max, int32_t* n_out);
/* Free a completed request's outputs in the arena. Thread-safe. */
ags_status ags_server_release(ags_server* server, uint64_t request_id);

/* Cancel a request that is still queued (not yet in a batch): it leaves the
 * queue and completes at once with status AGS_ERR_CANCELLED and no outputs.
 * AGS_ERR_BUSY if it is already batched, done or unknown. */
ags_status ags_server_cancel(ags_server* server, uint64_t request_id);
/* Counters; any pointer may be NULL. */
ags_status ags_server_stats(ags_server* server, int64_t* submitted, int64_t* completed, int64_t* batches,
                            int64_t* arena_free_bytes);
/* Load generator: submit reqs[i] at arrival_s[i] seconds after the call
 * starts (non-decreasing), collect every completion into out[i] and release
 * it; returns when all n are done. No other submissions may run meanwhile. */
ags_status ags_server_replay(ags_server* server, const ags_request* reqs, const double* arrival_s, int32_t n,
                             ags_completion* out);
/* Baseline for the same trace: one request at a time on the context's stream
 * (ags_render_envs of its environment, then synchronise), each started no
 * earlier than its arrival; out[i] as above (its buffers are freed on return). */
ags_status ags_replay_sequential(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* specs,
                                 int32_t n_specs, const ags_request* reqs, const double* arrival_s, int32_t n,
                                 ags_completion* out);

/*
 * Step graph: the render of one step (tile-counter reset + render kernel)
 * captured once as a CUDA graph over fixed buffers, then replayed with one
 * launch per step; the caller refreshes sensor_poses_dev between launches.
 * One graph must not run on two streams at once (they share its counter).
 * The graph holds the scene's device pointers: ags_scene_update_poses with
 * AGS_UPDATE_REFIT keeps it valid, AGS_UPDATE_REBUILD and ags_scene_destroy
 * invalidate it (destroy the graph first, then capture a new one). A launch
 * config set after capture applies to new graphs only. Errors: NULL or
 * mismatched handles and bad specs -> AGS_ERR_INVALID_ARG; capture or
 * instantiate failures -> AGS_ERR_CUDA. Device-side limits are reported by
 * ags_stream_status like any render. ags_render_graph_destroy synchronises
 * the device before freeing.
 */
typedef struct ags_graph ags_graph;
ags_status ags_render_graph_create(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* spec,
                                   const float* sensor_poses_dev, float* out_depth_dev, int32_t* out_seg_dev,
                                   ags_graph** out);
ags_status ags_render_graph_launch(ags_graph* graph, void* cuda_stream);
void ags_render_graph_destroy(ags_graph* graph);

/* Synchronise `cuda_stream`, then read and clear the context's device status
 * word: AGS_OK; AGS_ERR_INVALID_ARG if a device sensor pose was non-finite or
 * had a zero quaternion (those rays report NaN, segment -1);
 * AGS_ERR_TRAVERSAL_LIMIT if any ray since the last call hit a limit; or
 * AGS_ERR_CUDA. */
ags_status ags_stream_status(ags_context* ctx, void* cuda_stream);

/* Cap on the BVH nodes one ray may visit (default 1048576). A ray that reaches
 * it stops, reports NaN / segment -1 and makes the next ags_stream_status
 * return AGS_ERR_TRAVERSAL_LIMIT. Values below 1 are rejected. */
ags_status ags_context_set_traversal_cap(ags_context* ctx, int32_t max_node_visits);

/* Rays a short-stack render (ags_launch_config.stack_depth 16 or 32) may hand
 * to its full-stack retry pass, 0..1048576 (the default; the list's memory is
 * held by the context). Rays beyond it report NaN / segment -1 and make the
 * next ags_stream_status return AGS_ERR_TRAVERSAL_LIMIT. */
ags_status ags_context_set_retry_capacity(ags_context* ctx, int32_t rays);

/*
 * ags_transform_vertices_noalloc -- the object-to-world vertex transform of
 * ags_scene_build (v' = R(q) v + p per sub-mesh, float-float arithmetic, within
 * one unit in the last place) on caller-owned device buffers, without
 * allocating any memory. The paper has no counterpart: this entry point exists
 * for callers that cannot let a library call cudaMalloc -- a process whose
 * device memory is reserved up front by its own allocator (a fixed serving
 * memory plan, or a framework's caching allocator that owns the pool), or one
 * that cannot afford the device-wide synchronisation a cudaMalloc may cause in
 * the middle of its work.
 * base_vertices_dev: device float32 [n_vertices][3], object frames.
 * submesh_vertex_offsets_dev: device int32 [n_submeshes + 1], ascending, first
 *   0, last n_vertices; sub-mesh j owns vertices [off[j], off[j+1]).
 * poses_dev: device float32 [n_submeshes][7] (px, py, pz, qx, qy, qz, qw).
 * world_vertices_dev: device float32 [n_vertices][4], 16-byte aligned; xyz =
 *   world position, w = 0 (the layout the renderer keeps internally).
 * Asynchronous on cuda_stream. Its per-sub-mesh scratch (18 floats each) is a
 * fixed device array inside the library, sized for at most 65536 sub-meshes
 * (4.5 MiB, held by every GPU that loads the library until the process
 * exits); larger n_submeshes is rejected with AGS_ERR_INVALID_ARG. The first
 * call on a device looks up that array's device address (once per device),
 * so make that first call before any stream capture. All calls share the one
 * array: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller. Every scratch entry a call reads it first
 * writes, so nothing has to be cleared between calls. No device memory is
 * allocated; a successful call allocates no host memory either.
 */
ags_status ags_transform_vertices_noalloc(ags_context* ctx, const float* base_vertices_dev,
                                          int32_t n_vertices, const int32_t* submesh_vertex_offsets_dev,
                                          int32_t n_submeshes, const float* poses_dev,
                                          float* world_vertices_dev, void* cuda_stream);

/* Copy `bytes` from device memory to host memory (synchronous), e.g. a
 * completion's outputs. */
ags_status ags_memcpy_d2h(void* dst_host, const void* src_dev, int64_t bytes);

/* Thread-local text of the last error ("" if none). */
const char* ags_last_error(void);

/* Number of environments of a scene, or -1 for NULL. */
int32_t ags_scene_n_envs(const ags_scene* scene);

/*
 * ags_scene_get_world_triangles -- debug/test: the float32 world-space
 * triangles of environment `env` as the renderer sees them, in input order
 * (sub-mesh after sub-mesh): out_host [n][9] (x0 y0 z0 x1 y1 z1 x2 y2 z2) and
 * out_seg [n]; `capacity` is the number of rows the buffers hold, n the
 * environment's triangle count (ags_scene_stats).
 */
ags_status ags_scene_get_world_triangles(const ags_scene* scene, int32_t env, float* out_host,
                                         int32_t* out_seg, int64_t capacity);

/*
 * ags_scene_stats -- triangles, wide BVH nodes and resident bytes (nodes +
 * packed triangles, one 48-byte copy per BVH reference) of environment `env`,
 * or of the whole scene if env == -1.
 * Any output pointer may be NULL.
 */
ags_status ags_scene_stats(const ags_scene* scene, int32_t env, int64_t* n_tris, int64_t* n_nodes,
                           int64_t* bytes);

/* Size in bytes of one wide BVH node of the scene's format. */
int32_t ags_scene_node_bytes(const ags_scene* scene);

#ifdef __cplusplus
}
#endif
#endif /* AGS_H */
