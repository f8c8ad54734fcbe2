// ags_scene_validate: structural checks of a scene's BVH, on the host, from the
// device data the render kernel reads. Every environment's tree is walked
// from its root; the checks are the ones culling correctness rests on:
//   - every wide node is reached exactly once (no sharing, no cycles, none left out),
//     every reference exactly once, and every index is in range;
//   - each packed triangle copy equals its source triangle (vertices, segment ID,
//     environment-local index);
//   - every point of every triangle lies inside all boxes on the path to one of
//     its references (checked on a barycentric grid of points per triangle, in
//     double precision, on the decoded boxes of whatever node format the scene
//     uses), so a ray that meets a triangle reaches a leaf that holds it.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace ags {
namespace {

struct NodeInfo {
  int32_t child_base, tri_base;
  uint32_t meta_lo, meta_hi;
  double box[8][6];  // lo xyz, hi xyz
};

// the three node layouts, decoded to double boxes
struct HostF16 {
  int32_t child_base, tri_base;
  uint32_t meta_lo, meta_hi;
  float ox, oy, oz, pad;
  uint16_t v[6][8];  // lo_x, hi_x, lo_y, hi_y, lo_z, hi_z as float16 bits
};
struct HostQ8 {
  float ox, oy, oz;
  uint32_t exps;
  int32_t child_base, tri_base;
  uint32_t meta_lo, meta_hi;
  uint8_t v[6][8];
};
static_assert(sizeof(HostF16) == 128 && sizeof(HostQ8) == 80, "node layouts");

double half_bits(uint16_t h) {
  __half_raw r;
  r.x = h;
  return (double)__half2float(__half(r));
}

NodeInfo decode(const char* raw, int fmt) {
  NodeInfo n;
  if (fmt == kNodeFp32) {
    WideNode w;
    std::memcpy(&w, raw, sizeof(w));
    n.child_base = w.child_base;
    n.tri_base = w.tri_base;
    n.meta_lo = w.meta_lo;
    n.meta_hi = w.meta_hi;
    for (int k = 0; k < 8; ++k) {
      const double b[6] = {w.lox[k], w.loy[k], w.loz[k], w.hix[k], w.hiy[k], w.hiz[k]};
      std::memcpy(n.box[k], b, sizeof(b));
    }
  } else if (fmt == kNodeFp16) {
    HostF16 w;
    std::memcpy(&w, raw, sizeof(w));
    n.child_base = w.child_base;
    n.tri_base = w.tri_base;
    n.meta_lo = w.meta_lo;
    n.meta_hi = w.meta_hi;
    const double org[3] = {w.ox, w.oy, w.oz};
    for (int k = 0; k < 8; ++k)
      for (int a = 0; a < 3; ++a) {
        n.box[k][a] = org[a] + half_bits(w.v[2 * a][k]);
        n.box[k][3 + a] = org[a] + half_bits(w.v[2 * a + 1][k]);
      }
  } else {
    HostQ8 w;
    std::memcpy(&w, raw, sizeof(w));
    n.child_base = w.child_base;
    n.tri_base = w.tri_base;
    n.meta_lo = w.meta_lo;
    n.meta_hi = w.meta_hi;
    const double org[3] = {w.ox, w.oy, w.oz};
    for (int a = 0; a < 3; ++a) {
      const double scale = std::ldexp(1.0, (int)((w.exps >> (8 * a)) & 0xFFu) - 127);
      for (int k = 0; k < 8; ++k) {
        n.box[k][a] = org[a] + w.v[2 * a][k] * scale;
        n.box[k][3 + a] = org[a] + w.v[2 * a + 1][k] * scale;
      }
    }
  }
  return n;
}

uint32_t meta_of(const NodeInfo& n, int k) { return ((k < 4 ? n.meta_lo : n.meta_hi) >> (8 * (k & 3))) & 0xFFu; }

struct Checker {
  int64_t violations = 0;
  std::string first;
  void fail(const std::string& what) {
    if (violations++ < 4) first += (first.empty() ? "" : "; ") + what;
  }
};

// One level (a flat scene, or one level of a two-level scene). counts: nodes, points, violations, depth.
ags_status validate_level(const ags_scene* sc, Checker& chk, int64_t counts[4]) {
  cudaStream_t s = sc->ctx->stream;
  const int64_t N = sc->n_nodes, R = sc->n_refs, F = sc->n_tris, V = sc->n_verts;
  const int nb = node_bytes_of(sc->node_format);
  std::vector<char> raw((size_t)std::max<int64_t>(N, 1) * nb);
  std::vector<float4> tris((size_t)std::max<int64_t>(3 * R, 1)), verts((size_t)std::max<int64_t>(V, 1));
  std::vector<int32_t> root(sc->n_envs), leaf_tri((size_t)std::max<int64_t>(R, 1));
  std::vector<int32_t> vidx((size_t)std::max<int64_t>(3 * F, 1));
  cudaError_t e;
  if ((N > 0 &&
       (e = cudaMemcpyAsync(raw.data(), sc->d.nodes, (size_t)N * nb, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (R > 0 && (e = cudaMemcpyAsync(tris.data(), sc->d.tris, (size_t)(3 * R) * sizeof(float4), cudaMemcpyDeviceToHost,
                                     s)) != cudaSuccess) ||
      (R > 0 && (e = cudaMemcpyAsync(leaf_tri.data(), sc->d.leaf_tri, (size_t)R * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (V > 0 && (e = cudaMemcpyAsync(verts.data(), sc->d.world_verts, (size_t)V * sizeof(float4),
                                     cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (F > 0 && (e = cudaMemcpyAsync(vidx.data(), sc->d.tri_vidx, (size_t)(3 * F) * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (e = cudaMemcpyAsync(root.data(), sc->d.env_root, (size_t)sc->n_envs * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "validation read-back");

  // triangle -> environment and sub-mesh, for the copy checks
  std::vector<int32_t> tri_env((size_t)std::max<int64_t>(F, 1)), tri_sub((size_t)std::max<int64_t>(F, 1));
  for (int32_t en = 0; en < sc->n_envs; ++en)
    for (int64_t j = sc->env_sub_off[en]; j < sc->env_sub_off[en + 1]; ++j)
      for (int64_t t = sc->sub_tri_off[j]; t < sc->sub_tri_off[j + 1]; ++t) {
        tri_env[t] = en;
        tri_sub[t] = (int32_t)j;
      }

  std::vector<uint8_t> seen_node((size_t)std::max<int64_t>(N, 1), 0), seen_ref((size_t)std::max<int64_t>(R, 1), 0);
  std::vector<double> eff((size_t)std::max<int64_t>(R, 1) * 6);
  struct Item {
    int32_t node;
    int depth;
    double box[6];
  };
  std::vector<Item> stack;
  int64_t max_depth = 0;
  for (int32_t en = 0; en < sc->n_envs; ++en) {
    const int32_t r0 = root[en];
    if (r0 < 0) {
      if (sc->env_tri_off[en + 1] > sc->env_tri_off[en]) chk.fail("environment with triangles but no root");
      continue;
    }
    Item it{r0, 1, {-INFINITY, -INFINITY, -INFINITY, INFINITY, INFINITY, INFINITY}};
    stack.push_back(it);
    while (!stack.empty()) {
      Item cur = stack.back();
      stack.pop_back();
      if (cur.node < 0 || cur.node >= N) {
        chk.fail("node index out of range");
        continue;
      }
      if (seen_node[cur.node]++) {
        chk.fail("node reached twice");
        continue;
      }
      max_depth = std::max<int64_t>(max_depth, cur.depth);
      const NodeInfo n = decode(raw.data() + (size_t)cur.node * nb, sc->node_format);
      const uint32_t b0 = n.meta_lo & 0xFFu;
      const int ni = (b0 & 0x80u) ? (int)std::min(b0 & 0xFu, 8u) : 0;
      for (int k = 0; k < 8; ++k) {
        const uint32_t m = meta_of(n, k);
        if (m == kMetaEmpty) continue;
        double box[6];
        for (int a = 0; a < 3; ++a) {
          box[a] = std::max(cur.box[a], n.box[k][a]);
          box[3 + a] = std::min(cur.box[3 + a], n.box[k][3 + a]);
        }
        if (k < ni) {
          Item c{n.child_base + k, cur.depth + 1, {}};
          std::memcpy(c.box, box, sizeof(box));
          stack.push_back(c);
        } else {
          const int64_t start = (int64_t)n.tri_base + (m >> 2), cnt = (int64_t)(m & 3u) + 1;
          for (int64_t r = start; r < start + cnt; ++r) {
            if (r < 0 || r >= R) {
              chk.fail("reference index out of range");
              continue;
            }
            if (seen_ref[r]++) chk.fail("reference in two leaves");
            std::memcpy(&eff[6 * r], box, sizeof(box));
          }
        }
      }
    }
  }
  for (int64_t i = 0; i < N; ++i)
    if (!seen_node[i]) {
      chk.fail("node not reachable from its root");
      break;
    }
  // references: each copy equals its source triangle
  std::vector<std::vector<int32_t>> refs_of((size_t)std::max<int64_t>(F, 1));
  for (int64_t r = 0; r < R; ++r) {
    if (!seen_ref[r]) {
      chk.fail("reference in no leaf");
      continue;
    }
    const int32_t t = leaf_tri[r];
    if (t < 0 || t >= F) {
      chk.fail("reference of an unknown triangle");
      continue;
    }
    refs_of[t].push_back((int32_t)r);
    for (int c = 0; c < 3; ++c) {
      const float4 a = tris[3 * r + c], w = verts[vidx[3 * (int64_t)t + c]];
      if (a.x != w.x || a.y != w.y || a.z != w.z) chk.fail("packed triangle differs from its source");
    }
    int32_t seg, local;
    std::memcpy(&seg, &tris[3 * r].w, 4);
    std::memcpy(&local, &tris[3 * r + 1].w, 4);
    if (seg != sc->sub_seg[tri_sub[t]] || local != (int32_t)(t - sc->env_tri_off[tri_env[t]]))
      chk.fail("packed triangle's segment or index is wrong");
  }
  // coverage: points of every triangle inside the path boxes of one of its references
  const int G = 6;
  int64_t points = 0;
  for (int64_t t = 0; t < F; ++t) {
    if (refs_of[t].empty()) {
      chk.fail("triangle without a reference");
      continue;
    }
    double v[3][3];
    for (int c = 0; c < 3; ++c) {
      const float4 w = verts[vidx[3 * t + c]];
      v[c][0] = w.x;
      v[c][1] = w.y;
      v[c][2] = w.z;
    }
    for (int i = 0; i <= G; ++i)
      for (int j = 0; i + j <= G; ++j) {
        const double u = (double)i / G, w = (double)j / G;
        double p[3];
        for (int a = 0; a < 3; ++a) {
          // the exact point lies within the vertices' range; keep rounding from pushing it out
          // (a flat triangle's constant coordinate would otherwise drift by an ulp)
          const double lo = std::min(v[0][a], std::min(v[1][a], v[2][a]));
          const double hi = std::max(v[0][a], std::max(v[1][a], v[2][a]));
          p[a] = std::min(hi, std::max(lo, (1 - u - w) * v[0][a] + u * v[1][a] + w * v[2][a]));
        }
        bool in = false;
        for (int32_t r : refs_of[t]) {
          const double* b = &eff[6 * (int64_t)r];
          if (p[0] >= b[0] && p[1] >= b[1] && p[2] >= b[2] && p[0] <= b[3] && p[1] <= b[4] && p[2] <= b[5]) {
            in = true;
            break;
          }
        }
        ++points;
        if (!in) chk.fail("a point of a triangle lies outside every path to its references");
      }
  }
  counts[0] += N;
  counts[1] += points;
  counts[3] = std::max(counts[3], max_depth);
  return AGS_OK;
}

}  // namespace

}  // namespace ags

using namespace ags;

extern "C" ags_status ags_scene_validate(const ags_scene* sc, int64_t counts[4]) {
  try {
    if (!sc || !counts) {
      set_error("scene or counts is NULL");
      return AGS_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 4; ++k) counts[k] = 0;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(sc->ctx->device);
    Checker chk;
    ags_status st = AGS_OK;
    if (sc->objects) {
      st = validate_level(sc->objects, chk, counts);
      if (st == AGS_OK) st = validate_level(sc->top, chk, counts);
    } else {
      st = validate_level(sc, chk, counts);
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st != AGS_OK) return st;
    counts[2] = chk.violations;
    if (chk.violations) set_error(chk.first);
    return AGS_OK;
  } catch (const std::bad_alloc&) {
    set_error("out of host memory");
    return AGS_ERR_OUT_OF_MEMORY;
  } catch (...) {
    set_error("unexpected host exception");
    return AGS_ERR_CUDA;
  }
}
