// Serving: continuous batching of render requests over a resident scene.
//
// A worker thread takes requests in arrival order, admits as many as fit in
// the free part of a device output arena (and in a slot table), uploads their
// slot table and launches the render kernel in slot mode on one of several
// streams, so batches overlap on the GPU while new requests queue. A batch's
// requests complete together when its stream passes an event; their results
// stay in the arena (device memory, where a GPU consumer such as a policy
// network reads them) until the client releases them, which frees the space
// for later admissions.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace ags {
namespace {

constexpr int64_t kServerMaxPending = 1 << 20;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Pending {
  uint64_t id;
  ags_request req;
  double t_submit;
  int64_t elems;  // H * W of its sensor
};

struct InFlight {
  int lane = -1;  // which stream / staging set
  std::vector<Pending> reqs;
  std::vector<int64_t> offsets;  // arena element offsets
  double t_launch = 0;
  bool done = false;
};

struct Region {  // arena allocation, in allocation order
  uint64_t id;
  int64_t begin, end;
  bool released;
};

}  // namespace
}  // namespace ags

struct ags_server {
  ags_context* ctx = nullptr;
  const ags_scene* scene = nullptr;
  int32_t max_slots = 0, max_inflight = 0;
  std::vector<ags_sensor_spec> specs;
  std::vector<ags::SensorParams> params;
  ags::SensorParams* d_specs = nullptr;
  // arena: depth float32 and segment int32, same element offsets
  float* arena_depth = nullptr;
  int32_t* arena_seg = nullptr;
  int64_t arena_elems = 0;
  std::deque<ags::Region> regions;
  // per in-flight lane
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<ags::SlotEntry*> d_slots;
  std::vector<ags::SlotEntry*> h_slots;  // pinned staging
  std::vector<bool> lane_busy;
  std::vector<unsigned int*> counters;
  // use_graph: per lane, the batch step (slot-table copy, counter reset, render) as one captured graph whose
  // copy size is set per batch
  bool use_graph = false;
  std::vector<cudaGraph_t> graphs;
  std::vector<cudaGraphExec_t> gexec;
  std::vector<cudaGraphNode_t> gcopy;
  // queues
  std::mutex m;
  std::condition_variable cv;
  std::deque<ags::Pending> pending;
  std::deque<ags::InFlight> inflight;
  std::deque<ags_completion> done;
  uint64_t next_id = 1;
  int64_t submitted = 0, completed = 0, launched_batches = 0;
  bool auto_release = false;
  bool stop = false;
  int status_error = 0;
  std::thread worker;
};

namespace ags {
namespace {

// Ring allocation in request order: live regions run from the oldest one's
// start to the newest one's end, possibly wrapping past the arena's end.
bool arena_alloc(ags_server* sv, int64_t n, uint64_t id, int64_t* off) {
  const int64_t cap = sv->arena_elems;
  if (sv->regions.empty()) {
    if (n > cap) return false;
    *off = 0;
  } else {
    const int64_t tail = sv->regions.front().begin, head = sv->regions.back().end;
    if (head > tail) {  // live [tail, head): free [head, cap) and [0, tail)
      if (head + n <= cap) *off = head;
      else if (n <= tail) *off = 0;
      else return false;
    } else {  // wrapped, live [tail, cap) and [0, head): free [head, tail)
      if (head + n <= tail) *off = head;
      else return false;
    }
  }
  sv->regions.push_back({id, *off, *off + n, false});
  return true;
}

// Regions are in id order (admission is first in, first out), so a release
// finds its region by binary search; space returns once all older ones are
// released too.
void arena_release(ags_server* sv, uint64_t id) {
  auto it = std::lower_bound(sv->regions.begin(), sv->regions.end(), id,
                             [](const Region& r, uint64_t x) { return r.id < x; });
  if (it != sv->regions.end() && it->id == id) it->released = true;
  while (!sv->regions.empty() && sv->regions.front().released) sv->regions.pop_front();
}

void retire(ags_server* sv) {
  // completions in launch order per batch
  for (auto& b : sv->inflight) {
    if (b.done) continue;
    if (cudaEventQuery(sv->events[b.lane]) != cudaSuccess) continue;
    b.done = true;
    const double t = now_s();
    for (size_t k = 0; k < b.reqs.size(); ++k) {
      ags_completion c{};
      c.request_id = b.reqs[k].id;
      c.tag = b.reqs[k].req.tag;
      c.status = AGS_OK;
      c.depth_dev = sv->arena_depth + b.offsets[k];
      c.seg_dev = sv->arena_seg + b.offsets[k];
      c.t_submit = b.reqs[k].t_submit;
      c.t_start = b.t_launch;
      c.t_done = t;
      sv->done.push_back(c);
      ++sv->completed;
      if (sv->auto_release) arena_release(sv, c.request_id);
    }
    sv->lane_busy[b.lane] = false;
  }
  while (!sv->inflight.empty() && sv->inflight.front().done) sv->inflight.pop_front();
}

// The render arguments of one lane's batches: the slot table follows a
// one-entry header {n_slots, total_tiles} that the kernel reads from device
// memory, so the same arguments serve every batch (and a captured graph).
TraceArgs batch_args(ags_server* sv, int lane) {
  TraceArgs a{};
  a.nodes = sv->scene->d.nodes;
  a.node_format = sv->scene->node_format;
  a.tris = sv->scene->d.tris;
  a.env_root = sv->scene->d.env_root;
  a.n_nodes = (int32_t)sv->scene->n_nodes;
  a.n_tris = (int32_t)sv->scene->n_refs;
  a.n_scene_envs = sv->scene->n_envs;
  a.out_depth = sv->arena_depth;
  a.out_seg = sv->arena_seg;
  a.specs = sv->d_specs;
  a.n_specs = (int32_t)sv->params.size();
  a.slots = sv->d_slots[lane] + 1;
  a.slot_header = reinterpret_cast<const int32_t*>(sv->d_slots[lane]);
  a.n_slots = 0;
  a.log2_tile_w = 3;
  a.tile_h = 4;
  a.rays_per_lane = 1;
  a.total_tiles = 0;
  a.max_visits = sv->ctx->max_node_visits;
  a.status = sv->ctx->d_status;
  a.counts = sv->ctx->d_counts;
  a.tile_counter = sv->counters[lane];
  return a;
}

// Capture lane k's batch step into a graph (at server creation, before the worker starts).
cudaError_t capture_lane(ags_server* sv, int k) {
  cudaStream_t s = sv->streams[k];
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaMemcpyAsync(sv->d_slots[k], sv->h_slots[k], sizeof(SlotEntry), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(sv->counters[k], 0, sizeof(unsigned int), s);
  const cudaError_t le = launch_trace(batch_args(sv, k), sv->ctx->trace_blocks, false, s);
  e = cudaStreamEndCapture(s, &g);
  if (e == cudaSuccess && le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphNode_t copy = nullptr;
  if (e == cudaSuccess) {
    size_t n = 0;
    e = cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess) e = cudaGraphGetNodes(g, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      if (e == cudaSuccess && t == cudaGraphNodeTypeMemcpy) copy = nodes[i];
    }
    if (e == cudaSuccess && !copy) e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return e;
  }
  sv->graphs[k] = g;
  sv->gexec[k] = ge;
  sv->gcopy[k] = copy;
  return cudaSuccess;
}

bool launch_batch(ags_server* sv) {
  NvtxRange range("ags serving batch");
  int lane = -1;
  for (int k = 0; k < sv->max_inflight; ++k)
    if (!sv->lane_busy[k]) {
      lane = k;
      break;
    }
  if (lane < 0 || sv->pending.empty()) return false;
  InFlight b;
  b.lane = lane;
  int64_t tiles = 0;
  SlotEntry* hs = sv->h_slots[lane] + 1;  // entry 0 is the header
  while (!sv->pending.empty() && (int32_t)b.reqs.size() < sv->max_slots) {
    Pending& p = sv->pending.front();
    int64_t off = 0;
    if (!arena_alloc(sv, p.elems, p.id, &off)) break;  // admission: wait for free arena space
    const SensorParams& sp = sv->params[p.req.spec];
    SlotEntry& e = hs[b.reqs.size()];
    e.env = p.req.env;
    e.spec = p.req.spec;
    e.tile_begin = (int32_t)tiles;
    e.pad0 = 0;
    e.out_offset = off;
    std::memcpy(e.pose, p.req.pose, sizeof(e.pose));
    e.pad1 = 0.0f;
    tiles += sp.tiles_per_env;
    b.offsets.push_back(off);
    b.reqs.push_back(p);
    sv->pending.pop_front();
  }
  if (b.reqs.empty()) return false;
  cudaStream_t s = sv->streams[lane];
  const int n = (int)b.reqs.size();
  int32_t* hdr = reinterpret_cast<int32_t*>(sv->h_slots[lane]);
  hdr[0] = n;
  hdr[1] = (int32_t)tiles;
  const size_t bytes = (size_t)(n + 1) * sizeof(SlotEntry);
  if (sv->use_graph) {
    cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(sv->gexec[lane], sv->gcopy[lane], sv->d_slots[lane],
                                                       sv->h_slots[lane], bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaGraphLaunch(sv->gexec[lane], s);
    if (e != cudaSuccess) sv->status_error = 1;
  } else {
    cudaMemcpyAsync(sv->d_slots[lane], sv->h_slots[lane], bytes, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(sv->counters[lane], 0, sizeof(unsigned int), s);
    if (launch_trace(batch_args(sv, lane), sv->ctx->trace_blocks, false, s) != cudaSuccess) sv->status_error = 1;
  }
  cudaEventRecord(sv->events[lane], s);
  b.t_launch = now_s();
  sv->lane_busy[lane] = true;
  sv->inflight.push_back(std::move(b));
  ++sv->launched_batches;
  return true;
}

void worker_main(ags_server* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->m);
  while (true) {
    retire(sv);
    bool launched = false;
    while (launch_batch(sv)) launched = true;
    if (sv->stop && sv->pending.empty() && sv->inflight.empty()) break;
    if (!launched) {
      if (sv->inflight.empty() && sv->pending.empty())
        sv->cv.wait(lk, [&] { return sv->stop || !sv->pending.empty(); });
      else
        sv->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

ags_status invalid_arg(const char* msg) {
  set_error(msg);
  return AGS_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace ags

using namespace ags;

extern "C" {

ags_status ags_server_create(ags_context* ctx, const ags_scene* scene, const ags_server_config* cfg,
                             ags_server** out) {
  try {
    if (!out) return invalid_arg("out is NULL");
    *out = nullptr;
    if (!ctx || !scene || !cfg) return invalid_arg("ctx, scene or config is NULL");
    if (scene->ctx != ctx) return invalid_arg("scene belongs to another context");
    if (scene->objects) return invalid_arg("serving needs a single-level scene");
    if (cfg->max_slots < 1 || cfg->max_slots > 65536) return invalid_arg("max_slots must be in [1, 65536]");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 16) return invalid_arg("max_inflight must be in [1, 16]");
    if (cfg->n_specs < 1 || cfg->n_specs > 256 || !cfg->specs) return invalid_arg("need 1..256 sensor specs");
    cudaSetDevice(ctx->device);
    std::unique_ptr<ags_server> sv(new ags_server());
    sv->ctx = ctx;
    sv->scene = scene;
    sv->max_slots = cfg->max_slots;
    sv->max_inflight = cfg->max_inflight;
    sv->auto_release = cfg->auto_release != 0;
    int64_t max_req = 0;
    for (int32_t k = 0; k < cfg->n_specs; ++k) {
      const ags_sensor_spec& s = cfg->specs[k];
      if (s.type != AGS_PINHOLE && s.type != AGS_LIDAR) return invalid_arg("spec type invalid");
      if (s.width < 1 || s.width > 16384 || s.height < 1 || s.height > 16384) return invalid_arg("spec size invalid");
      if (!(s.max_range > s.min_range) || s.min_range < 0.0f || s.flags != 0) return invalid_arg("spec ranges invalid");
      sv->specs.push_back(s);
      sv->params.push_back(sensor_params(&s, 8, 4));
      max_req = std::max<int64_t>(max_req, (int64_t)s.width * s.height);
    }
    // arena: the requested bytes, limited by what the device has free now
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    int64_t want = cfg->arena_bytes > 0 ? cfg->arena_bytes : (int64_t)(free_b / 4);
    want = std::min<int64_t>(want, (int64_t)(free_b * 0.9));
    sv->arena_elems = want / 8;
    if (sv->arena_elems < max_req) return invalid_arg("arena cannot hold one request of the largest sensor");
    if ((e = cudaMalloc(&sv->arena_depth, sv->arena_elems * sizeof(float))) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc(arena)");
    if ((e = cudaMalloc(&sv->arena_seg, sv->arena_elems * sizeof(int32_t))) != cudaSuccess) {
      cudaFree(sv->arena_depth);
      return cuda_fail(e, "cudaMalloc(arena)");
    }
    if ((e = cudaMalloc(&sv->d_specs, sv->params.size() * sizeof(SensorParams))) != cudaSuccess ||
        (e = cudaMemcpy(sv->d_specs, sv->params.data(), sv->params.size() * sizeof(SensorParams),
                        cudaMemcpyHostToDevice)) != cudaSuccess) {
      cudaFree(sv->arena_depth);
      cudaFree(sv->arena_seg);
      return cuda_fail(e, "spec table");
    }
    for (int k = 0; k < sv->max_inflight; ++k) {
      cudaStream_t s;
      cudaEvent_t ev;
      SlotEntry *ds, *hs;
      if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaMalloc(&ds, (sv->max_slots + 1) * sizeof(SlotEntry))) != cudaSuccess ||
          (e = cudaHostAlloc(&hs, (sv->max_slots + 1) * sizeof(SlotEntry), cudaHostAllocDefault)) != cudaSuccess) {
        ags_server* raw = sv.release();
        ags_server_destroy(raw);
        return cuda_fail(e, "server lane setup");
      }
      sv->streams.push_back(s);
      sv->events.push_back(ev);
      sv->d_slots.push_back(ds);
      sv->h_slots.push_back(hs);
      sv->lane_busy.push_back(false);
      unsigned int* counter = nullptr;
      if ((e = cudaMalloc(&counter, sizeof(unsigned int))) != cudaSuccess) {
        ags_server* raw = sv.release();
        ags_server_destroy(raw);
        return cuda_fail(e, "server tile counter");
      }
      sv->counters.push_back(counter);
    }
    sv->use_graph = cfg->use_graph != 0;
    sv->graphs.assign(sv->max_inflight, nullptr);
    sv->gexec.assign(sv->max_inflight, nullptr);
    sv->gcopy.assign(sv->max_inflight, nullptr);
    if (sv->use_graph) {
      for (int k = 0; k < sv->max_inflight; ++k) {
        std::memset(sv->h_slots[k], 0, sizeof(SlotEntry));
        if ((e = capture_lane(sv.get(), k)) != cudaSuccess) {
          ags_server* raw = sv.release();
          ags_server_destroy(raw);
          return cuda_fail(e, "server graph capture");
        }
      }
    }
    ags_server* raw = sv.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return AGS_OK;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return AGS_ERR_OUT_OF_MEMORY;
  } catch (...) {
    set_error("unexpected host exception");
    return AGS_ERR_CUDA;
  }
}

void ags_server_destroy(ags_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->m);
    sv->stop = true;
    sv->pending.clear();
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->ctx->device);
  for (size_t k = 0; k < sv->streams.size(); ++k) cudaStreamSynchronize(sv->streams[k]);
  for (size_t k = 0; k < sv->gexec.size(); ++k) {
    if (sv->gexec[k]) cudaGraphExecDestroy(sv->gexec[k]);
    if (sv->graphs[k]) cudaGraphDestroy(sv->graphs[k]);
  }
  for (size_t k = 0; k < sv->streams.size(); ++k) {
    if (k < sv->counters.size()) cudaFree(sv->counters[k]);
    cudaStreamDestroy(sv->streams[k]);
    cudaEventDestroy(sv->events[k]);
    cudaFree(sv->d_slots[k]);
    cudaFreeHost(sv->h_slots[k]);
  }
  cudaFree(sv->arena_depth);
  cudaFree(sv->arena_seg);
  cudaFree(sv->d_specs);
  delete sv;
}

ags_status ags_server_submit(ags_server* sv, const ags_request* req, uint64_t* request_id) {
  if (!sv || !req) return invalid_arg("server or request is NULL");
  if (req->env < 0 || req->env >= sv->scene->n_envs) return invalid_arg("request env out of range");
  if (req->spec < 0 || req->spec >= (int32_t)sv->specs.size()) return invalid_arg("request spec out of range");
  for (int k = 0; k < 7; ++k)
    if (!std::isfinite(req->pose[k])) return invalid_arg("request pose not finite");
  const ags_sensor_spec& s = sv->specs[req->spec];
  const int64_t elems = (int64_t)s.width * s.height;
  {
    std::lock_guard<std::mutex> lk(sv->m);
    if (sv->stop) return invalid_arg("server is stopping");
    if (sv->pending.size() >= (size_t)kServerMaxPending) {
      set_error("request queue full");
      return AGS_ERR_BUSY;
    }
    ags::Pending p{sv->next_id++, *req, now_s(), elems};
    sv->pending.push_back(p);
    ++sv->submitted;
    if (request_id) *request_id = p.id;
  }
  sv->cv.notify_one();
  return AGS_OK;
}

ags_status ags_server_poll(ags_server* sv, ags_completion* out, int32_t max, int32_t* n_out) {
  if (!sv || !n_out || (max > 0 && !out)) return invalid_arg("server, out or n_out is NULL");
  std::lock_guard<std::mutex> lk(sv->m);
  int32_t n = 0;
  while (n < max && !sv->done.empty()) {
    out[n++] = sv->done.front();
    sv->done.pop_front();
  }
  *n_out = n;
  if (sv->status_error) {
    set_error("a serving batch failed to launch");
    return AGS_ERR_CUDA;
  }
  return AGS_OK;
}

ags_status ags_server_release(ags_server* sv, uint64_t request_id) {
  if (!sv) return invalid_arg("server is NULL");
  {
    std::lock_guard<std::mutex> lk(sv->m);
    arena_release(sv, request_id);
  }
  sv->cv.notify_one();
  return AGS_OK;
}

ags_status ags_server_cancel(ags_server* sv, uint64_t request_id) {
  if (!sv) return invalid_arg("server is NULL");
  std::lock_guard<std::mutex> lk(sv->m);
  for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it) {
    if (it->id != request_id) continue;
    ags_completion c{};
    c.request_id = it->id;
    c.tag = it->req.tag;
    c.status = AGS_ERR_CANCELLED;
    c.t_submit = it->t_submit;
    c.t_start = c.t_done = now_s();
    sv->pending.erase(it);
    sv->done.push_back(c);
    ++sv->completed;
    return AGS_OK;
  }
  set_error("request is not queued (already batched, done or unknown)");
  return AGS_ERR_BUSY;
}

ags_status ags_server_stats(ags_server* sv, int64_t* submitted, int64_t* completed, int64_t* batches,
                            int64_t* arena_free_bytes) {
  if (!sv) return invalid_arg("server is NULL");
  std::lock_guard<std::mutex> lk(sv->m);
  if (submitted) *submitted = sv->submitted;
  if (completed) *completed = sv->completed;
  if (batches) *batches = sv->launched_batches;
  if (arena_free_bytes) {
    int64_t live = 0;
    for (auto& r : sv->regions) live += r.end - r.begin;
    *arena_free_bytes = (sv->arena_elems - live) * 8;
  }
  return AGS_OK;
}

ags_status ags_server_replay(ags_server* sv, const ags_request* reqs, const double* arrival_s, int32_t n,
                             ags_completion* out) {
  if (!sv || (n > 0 && (!reqs || !arrival_s || !out))) return invalid_arg("NULL argument");
  if (n < 0) return invalid_arg("n < 0");
  std::vector<uint64_t> ids(n);
  uint64_t first_id;
  {
    std::lock_guard<std::mutex> lk(sv->m);
    first_id = sv->next_id;
  }
  const double t0 = now_s();
  int32_t next = 0, got = 0;
  std::vector<ags_completion> buf(256);
  while (got < n) {
    const double t = now_s() - t0;
    while (next < n && arrival_s[next] <= t) {
      ags_status st = ags_server_submit(sv, &reqs[next], &ids[next]);
      if (st != AGS_OK) return st;
      ++next;
    }
    int32_t k = 0;
    ags_status st = ags_server_poll(sv, buf.data(), (int32_t)buf.size(), &k);
    if (st != AGS_OK) return st;
    for (int32_t i = 0; i < k; ++i) {
      const uint64_t id = buf[i].request_id;
      if (id < first_id || id >= first_id + (uint64_t)n) continue;
      out[id - first_id] = buf[i];
      ++got;
      if (!sv->auto_release) ags_server_release(sv, id);
    }
    if (k == 0) {
      if (next < n && arrival_s[next] - (now_s() - t0) > 200e-6)
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      else
        std::this_thread::yield();
    }
  }
  return AGS_OK;
}

ags_status ags_replay_sequential(ags_context* ctx, const ags_scene* scene, const ags_sensor_spec* specs,
                                 int32_t n_specs, const ags_request* reqs, const double* arrival_s, int32_t n,
                                 ags_completion* out) {
  if (!ctx || !scene || !specs || n_specs < 1 || (n > 0 && (!reqs || !arrival_s || !out)))
    return invalid_arg("NULL argument");
  cudaSetDevice(ctx->device);
  int64_t max_el = 0;
  for (int32_t k = 0; k < n_specs; ++k) max_el = std::max<int64_t>(max_el, (int64_t)specs[k].width * specs[k].height);
  float* d_depth = nullptr;
  int32_t *d_seg = nullptr, *d_env = nullptr;
  float* d_pose = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&d_depth, max_el * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&d_seg, max_el * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&d_env, sizeof(int32_t))) != cudaSuccess || (e = cudaMalloc(&d_pose, 7 * sizeof(float))) != cudaSuccess) {
    cudaFree(d_depth);
    cudaFree(d_seg);
    cudaFree(d_env);
    return cuda_fail(e, "sequential replay buffers");
  }
  cudaStream_t s = ctx->stream;
  const double t0 = now_s();
  ags_status st = AGS_OK;
  for (int32_t i = 0; i < n && st == AGS_OK; ++i) {
    while (now_s() - t0 < arrival_s[i]) std::this_thread::yield();
    const double t_start = now_s();
    const ags_request& r = reqs[i];
    if (r.spec < 0 || r.spec >= n_specs) {
      st = invalid_arg("request spec out of range");
      break;
    }
    cudaMemcpyAsync(d_env, &r.env, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_pose, r.pose, 7 * sizeof(float), cudaMemcpyHostToDevice, s);
    st = ags_render_envs(ctx, scene, &specs[r.spec], d_env, 1, d_pose, d_depth, d_seg, s);
    if (st == AGS_OK) st = ags_stream_status(ctx, s);
    ags_completion c{};
    c.request_id = (uint64_t)i;
    c.tag = r.tag;
    c.status = st;
    c.depth_dev = d_depth;
    c.seg_dev = d_seg;
    c.t_submit = t0 + arrival_s[i];
    c.t_start = t_start;
    c.t_done = now_s();
    out[i] = c;
  }
  cudaFree(d_depth);
  cudaFree(d_seg);
  cudaFree(d_env);
  cudaFree(d_pose);
  return st;
}

}  // extern "C"
