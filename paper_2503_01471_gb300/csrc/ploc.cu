// Binary BVH by parallel locally-ordered clustering (Meister and Bittner,
// "Parallel Locally-Ordered Clustering for Bounding Volume Hierarchy
// Construction", IEEE TVCG 2018), per environment, all environments at once.
// The paper's method only says that a BVH is built for each environment's
// meshes (Sec. III-D.1); this builder gives a tree of lower surface-area cost
// than the Morton radix tree, so traversal visits fewer nodes.
//
// The references arrive sorted environment-major by Morton code. Each round,
// every cluster finds the cluster within `kRadius` positions (same
// environment) whose union box has the smallest surface area; mutual nearest
// pairs merge into a new inner node; the survivors are compacted in order.
// Rounds repeat until each environment is one cluster. The search radius is a
// build option (16 by default; 32, 64 or 128): a wider search finds better
// pairs at a proportional cost per round. The tree is then laid
// out for the wide-node collapse: leaves reordered depth-first so that every
// subtree covers a contiguous range of positions (first/last), as in a
// Morton radix tree.
#include "internal.cuh"

namespace ags {
namespace {

constexpr int kPlocThreads = 256;

__device__ __forceinline__ Box box_join(const Box& a, const Box& b) {
  return {fminf(a.lox, b.lox), fminf(a.loy, b.loy), fminf(a.loz, b.loz),
          fmaxf(a.hix, b.hix), fmaxf(a.hiy, b.hiy), fmaxf(a.hiz, b.hiz)};
}

__device__ __forceinline__ float half_area(const Box& b) {
  const float dx = b.hix - b.lox, dy = b.hiy - b.loy, dz = b.hiz - b.loz;
  return dx * dy + dy * dz + dz * dx;
}

__global__ void k_ploc_init(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int32_t R,
                            int key_shift, const Box* __restrict__ ref_box, int32_t* __restrict__ c_ref,
                            Box* __restrict__ c_box, int32_t* __restrict__ c_env) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R) return;
  c_ref[i] = ~i;
  c_box[i] = ref_box[vals[i]];
  c_env[i] = (int32_t)(keys[i] >> key_shift);
}

// Nearest neighbour of each cluster among the kRadius positions on either
// side in the same environment, by the surface area of the union box; ties
// go to the smaller position, so the globally closest pair is always mutual.
template <int kRadius>
__global__ void __launch_bounds__(kPlocThreads) k_ploc_nn(const Box* __restrict__ c_box,
                                                          const int32_t* __restrict__ c_env, int32_t n,
                                                          int32_t* __restrict__ nn) {
  __shared__ Box sb[kPlocThreads + 2 * kRadius];
  __shared__ int32_t se[kPlocThreads + 2 * kRadius];
  const int32_t b0 = (int32_t)blockIdx.x * kPlocThreads - kRadius;
  for (int k = threadIdx.x; k < kPlocThreads + 2 * kRadius; k += kPlocThreads) {
    const int32_t g = b0 + k;
    if (g >= 0 && g < n) {
      sb[k] = c_box[g];
      se[k] = c_env[g];
    } else {
      se[k] = -1;
    }
  }
  __syncthreads();
  const int32_t i = (int32_t)blockIdx.x * kPlocThreads + threadIdx.x;
  if (i >= n) return;
  const int li = threadIdx.x + kRadius;
  const Box bi = sb[li];
  const int32_t ei = se[li];
  float best = INFINITY;
  int32_t bj = -1;
#pragma unroll 4
  for (int o = -kRadius; o <= kRadius; ++o) {
    if (o == 0 || se[li + o] != ei) continue;
    const float d = half_area(box_join(bi, sb[li + o]));
    if (d < best) {
      best = d;
      bj = i + o;
    }
  }
  nn[i] = bj;
}

__device__ __forceinline__ bool mutual_lead(const int32_t* nn, int32_t i) {
  const int32_t j = nn[i];
  return j > i && nn[j] == i;
}
__device__ __forceinline__ bool absorbed(const int32_t* nn, int32_t i) {
  const int32_t j = nn[i];
  return j >= 0 && j < i && nn[j] == i;
}

__global__ void k_ploc_flag(const int32_t* __restrict__ nn, int32_t n, int32_t* __restrict__ flag) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = mutual_lead(nn, i) ? 1 : 0;
}

// Mutual pairs become inner nodes node_base + rank; every cluster's
// successor (new node, itself, or nothing when absorbed) is written out.
__global__ void k_ploc_merge(const int32_t* __restrict__ nn, int32_t n, const int32_t* __restrict__ c_ref,
                             const Box* __restrict__ c_box, const int32_t* __restrict__ rank, int32_t node_base,
                             int32_t node_cap, int32_t* __restrict__ left, int32_t* __restrict__ right,
                             Box* __restrict__ inner_box, int32_t* __restrict__ node_size,
                             int32_t* __restrict__ keep, int32_t* __restrict__ n_ref, Box* __restrict__ n_box,
                             int* __restrict__ err) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mutual_lead(nn, i)) {
    const int32_t j = nn[i];
    const int32_t id = node_base + rank[i];
    if (id < 0 || id >= node_cap) {
      atomicOr(err, 1);
      keep[i] = 0;
      return;
    }
    const int32_t a = c_ref[i], b = c_ref[j];
    const Box u = box_join(c_box[i], c_box[j]);
    left[id] = a;
    right[id] = b;
    inner_box[id] = u;
    node_size[id] = (a >= 0 ? node_size[a] : 1) + (b >= 0 ? node_size[b] : 1);
    n_ref[i] = id;
    n_box[i] = u;
    keep[i] = 1;
  } else if (absorbed(nn, i)) {
    keep[i] = 0;
  } else {
    n_ref[i] = c_ref[i];
    n_box[i] = c_box[i];
    keep[i] = 1;
  }
}

__global__ void k_ploc_compact(const int32_t* __restrict__ nn, int32_t n, const int32_t* __restrict__ pos,
                               const int32_t* __restrict__ n_ref, const Box* __restrict__ n_box,
                               const int32_t* __restrict__ c_env, int32_t* __restrict__ o_ref,
                               Box* __restrict__ o_box, int32_t* __restrict__ o_env) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || absorbed(nn, i)) return;
  const int32_t p = pos[i];
  o_ref[p] = n_ref[i];
  o_box[p] = n_box[i];
  o_env[p] = c_env[i];
}

// The last cluster of each environment is its root; it starts at the
// environment's first position.
__global__ void k_ploc_roots(const int32_t* __restrict__ c_ref, const int32_t* __restrict__ c_env, int32_t n,
                             int32_t E, int32_t R, const int32_t* __restrict__ env_ref_off,
                             int32_t* __restrict__ first, int32_t* __restrict__ newpos, int32_t* __restrict__ roots,
                             int32_t n_inner, int* __restrict__ err) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int32_t e = c_env[k], r = c_ref[k];
  if (e < 0 || e >= E) {
    atomicOr(err, 1);
    return;
  }
  roots[e] = r;
  const int32_t base = env_ref_off[e];
  if (r >= 0 && r < n_inner) first[r] = base;
  else if (r < 0 && ~r < R) newpos[~r] = base;
  else atomicOr(err, 1);
}

// Depth-first ranges, one round's nodes at a time from the last round back
// (a node's parent is always made in a later round than the node).
__global__ void k_ploc_down(int32_t b, int32_t e, const int32_t* __restrict__ left,
                            const int32_t* __restrict__ right, const int32_t* __restrict__ node_size, int32_t R,
                            int32_t* __restrict__ first, int32_t* __restrict__ last, int32_t* __restrict__ newpos,
                            int* __restrict__ err) {
  const int32_t id = b + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (id >= e) return;
  const int32_t f = first[id];
  const int32_t l = left[id], r = right[id];
  const int32_t sl = l >= 0 ? node_size[l] : 1;
  if (f < 0 || f + node_size[id] > R || l >= id || r >= id || (l < 0 && ~l >= R) || (r < 0 && ~r >= R)) {
    atomicOr(err, 1);
    return;
  }
  if (l >= 0) first[l] = f; else newpos[~l] = f;
  if (r >= 0) first[r] = f + sl; else newpos[~r] = f + sl;
  last[id] = f + node_size[id] - 1;
}

__global__ void k_ploc_remap(int32_t R, const int32_t* __restrict__ newpos, const uint32_t* __restrict__ vals,
                             const Box* __restrict__ ref_box, uint32_t* __restrict__ vals_out,
                             Box* __restrict__ leaf_box, int* __restrict__ err) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= R) return;
  const int32_t q = newpos[p];
  if (q < 0 || q >= R) {
    atomicOr(err, 1);
    return;
  }
  vals_out[q] = vals[p];
  leaf_box[q] = ref_box[vals[p]];
}

__global__ void k_ploc_relabel(int32_t n_inner, int32_t R, int32_t* __restrict__ left, int32_t* __restrict__ right,
                               const int32_t* __restrict__ newpos) {
  const int32_t id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_inner) return;
  const int32_t l = left[id], r = right[id];
  if (l < 0 && ~l < R) left[id] = ~newpos[~l];
  if (r < 0 && ~r < R) right[id] = ~newpos[~r];
}

// ---- wide-node slots of least surface-area cost (the collapse's choice)
// Cost of a wide tree under the surface-area heuristic: a ray that enters a
// box of area A' enters a child box of area A with probability A / A', so a
// wide node costs kCostNode * A (its eight child tests) and a leaf of c
// references kCostTri * c * A (its triangle tests). For an inner node n of
// the binary tree and a budget of i = 1..8 slots of one wide node, D(n, i) is
// the least cost of covering n's subtree with at most i slots:
//   D(n, 1) = kCostTri * c(n) * A(n)          when c(n) <= leaf_max (a leaf)
//           = kCostNode * A(n) + S(n, 8)      otherwise (a wide node of its own)
//   S(n, i) = min over k = 1..i-1 of D(left, k) + D(right, i - k)
//   D(n, i) = min(D(n, 1), S(n, i))           for i >= 2
// (a single reference is a leaf slot at every budget). Children are made in
// earlier clustering rounds than their parent, so the rounds in order give a
// bottom-up pass. choice[n] packs, for i = 2..8, the k of S(n, i) less one
// (3 bits at 3 (i - 2)) and whether D(n, i) keeps n as one slot (bit 21 + i - 2).
constexpr float kCostNode = kSahNodeCost, kCostTri = kSahTriCost;

__global__ void k_collapse_cost(int32_t b, int32_t e, const int32_t* __restrict__ left,
                                const int32_t* __restrict__ right, const int32_t* __restrict__ first,
                                const int32_t* __restrict__ last, const Box* __restrict__ inner_box,
                                const Box* __restrict__ leaf_box, int leaf_max, float* __restrict__ cost,
                                uint32_t* __restrict__ choice) {
  const int32_t id = b + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (id >= e) return;
  float dl[8], dr[8];
  const int32_t l = left[id], r = right[id];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    dl[k] = l >= 0 ? cost[8 * (int64_t)l + k] : kCostTri * half_area(leaf_box[~l]);
    dr[k] = r >= 0 ? cost[8 * (int64_t)r + k] : kCostTri * half_area(leaf_box[~r]);
  }
  float split[9];
  uint32_t ch = 0;
#pragma unroll
  for (int i = 2; i <= 8; ++i) {
    float best = INFINITY;
    int bk = 1;
#pragma unroll
    for (int k = 1; k < i; ++k) {
      const float c = dl[k - 1] + dr[i - k - 1];
      if (c < best) {
        best = c;
        bk = k;
      }
    }
    split[i] = best;
    ch |= (uint32_t)(bk - 1) << (3 * (i - 2));
  }
  const int32_t cnt = last[id] - first[id] + 1;
  const float area = half_area(inner_box[id]);
  const float one = cnt <= leaf_max ? kCostTri * (float)cnt * area : kCostNode * area + split[8];
  cost[8 * (int64_t)id] = one;
#pragma unroll
  for (int i = 2; i <= 8; ++i) {
    const bool keep = one <= split[i];
    cost[8 * (int64_t)id + i - 1] = keep ? one : split[i];
    ch |= keep ? (1u << (21 + i - 2)) : 0u;
  }
  choice[id] = ch;
}

int blocks_of(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

ags_status build_ploc(const uint64_t* keys, uint32_t* vals, int32_t R, int key_shift, const int32_t* env_ref_off,
                      int32_t E, const Box* ref_box, Box* leaf_box, int32_t* left, int32_t* right, int32_t* first,
                      int32_t* last, Box* inner_box, std::vector<int32_t>& roots, cudaStream_t s,
                      uint32_t* choice, int leaf_max, int radius) {
  if (radius != 16 && radius != 32 && radius != 64 && radius != 128) {
    set_error("clustering radius must be 16, 32, 64 or 128");
    return AGS_ERR_INVALID_ARG;
  }
  NvtxRange range("ags clustering");
  roots.assign(E, -1);
  if (R <= 0) return AGS_OK;
  DevBufs tmp;
  int32_t *c_ref[2], *c_env[2], *nn, *flag, *keep, *n_ref, *node_size, *newpos, *d_roots, *d_tot;
  Box *c_box[2], *n_box;
  uint32_t* vals2;
  int* err;
  for (int k = 0; k < 2; ++k) {
    AGS_CHECK(tmp.alloc(&c_ref[k], (size_t)R));
    AGS_CHECK(tmp.alloc(&c_env[k], (size_t)R));
    AGS_CHECK(tmp.alloc(&c_box[k], (size_t)R));
  }
  AGS_CHECK(tmp.alloc(&nn, (size_t)R));
  AGS_CHECK(tmp.alloc(&flag, (size_t)R));
  AGS_CHECK(tmp.alloc(&keep, (size_t)R));
  AGS_CHECK(tmp.alloc(&n_ref, (size_t)R));
  AGS_CHECK(tmp.alloc(&n_box, (size_t)R));
  AGS_CHECK(tmp.alloc(&node_size, (size_t)R));
  AGS_CHECK(tmp.alloc(&newpos, (size_t)R));
  AGS_CHECK(tmp.alloc(&d_roots, (size_t)E));
  AGS_CHECK(tmp.alloc(&d_tot, 2));
  AGS_CHECK(tmp.alloc(&vals2, (size_t)R));
  AGS_CHECK(tmp.alloc(&err, 1));
  void* scan_tmp = nullptr;
  AGS_CHECK(tmp.alloc(reinterpret_cast<char**>(&scan_tmp), scan_temp_bytes(R)));
  AGS_CHECK(cudaMemsetAsync(err, 0, sizeof(int), s));
  AGS_CHECK(cudaMemsetAsync(d_roots, 0xFF, (size_t)E * sizeof(int32_t), s));
  AGS_CHECK(cudaMemsetAsync(first, 0xFF, (size_t)R * sizeof(int32_t), s));
  AGS_CHECK(cudaMemsetAsync(newpos, 0xFF, (size_t)R * sizeof(int32_t), s));

  k_ploc_init<<<blocks_of(R, 256), 256, 0, s>>>(keys, vals, R, key_shift, ref_box, c_ref[0], c_box[0], c_env[0]);
  AGS_CHECK(cudaGetLastError());
  int cur = 0;
  int32_t n = R, node_base = 0;
  std::vector<std::pair<int32_t, int32_t>> rounds;
  for (int it = 0;; ++it) {
    if (it > 4096) {
      set_error("clustering did not terminate");
      return AGS_ERR_CUDA;
    }
    const int nb = blocks_of(n, kPlocThreads);
    if (radius == 16) k_ploc_nn<16><<<nb, kPlocThreads, 0, s>>>(c_box[cur], c_env[cur], n, nn);
    else if (radius == 32) k_ploc_nn<32><<<nb, kPlocThreads, 0, s>>>(c_box[cur], c_env[cur], n, nn);
    else if (radius == 64) k_ploc_nn<64><<<nb, kPlocThreads, 0, s>>>(c_box[cur], c_env[cur], n, nn);
    else k_ploc_nn<128><<<nb, kPlocThreads, 0, s>>>(c_box[cur], c_env[cur], n, nn);
    k_ploc_flag<<<blocks_of(n, 256), 256, 0, s>>>(nn, n, flag);
    AGS_CHECK(cudaGetLastError());
    AGS_CHECK(exclusive_scan(flag, n, d_tot, scan_tmp, s));
    int32_t m = 0;
    AGS_CHECK(cudaMemcpyAsync(&m, d_tot, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AGS_CHECK(cudaStreamSynchronize(s));
    if (m < 0 || m > n / 2 || (int64_t)node_base + m > R) {
      set_error("clustering produced an inconsistent merge count");
      return AGS_ERR_CUDA;
    }
    if (m == 0) break;
    k_ploc_merge<<<blocks_of(n, 256), 256, 0, s>>>(nn, n, c_ref[cur], c_box[cur], flag, node_base, R, left, right,
                                                  inner_box, node_size, keep, n_ref, n_box, err);
    AGS_CHECK(cudaGetLastError());
    AGS_CHECK(exclusive_scan(keep, n, d_tot + 1, scan_tmp, s));
    k_ploc_compact<<<blocks_of(n, 256), 256, 0, s>>>(nn, n, keep, n_ref, n_box, c_env[cur], c_ref[1 - cur],
                                                    c_box[1 - cur], c_env[1 - cur]);
    AGS_CHECK(cudaGetLastError());
    rounds.push_back({node_base, node_base + m});
    node_base += m;
    n -= m;
    cur = 1 - cur;
  }
  const int32_t n_inner = node_base;
  k_ploc_roots<<<blocks_of(n, 256), 256, 0, s>>>(c_ref[cur], c_env[cur], n, E, R, env_ref_off, first, newpos, d_roots,
                                                n_inner, err);
  for (size_t k = rounds.size(); k-- > 0;) {
    const int32_t b = rounds[k].first, e = rounds[k].second;
    k_ploc_down<<<blocks_of(e - b, 256), 256, 0, s>>>(b, e, left, right, node_size, R, first, last, newpos, err);
  }
  k_ploc_remap<<<blocks_of(R, 256), 256, 0, s>>>(R, newpos, vals, ref_box, vals2, leaf_box, err);
  if (n_inner > 0) k_ploc_relabel<<<blocks_of(n_inner, 256), 256, 0, s>>>(n_inner, R, left, right, newpos);
  AGS_CHECK(cudaGetLastError());
  AGS_CHECK(cudaMemcpyAsync(vals, vals2, (size_t)R * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  if (choice && n_inner > 0) {
    float* cost = nullptr;
    AGS_CHECK(tmp.alloc(&cost, 8 * (size_t)n_inner));
    for (const auto& rd : rounds)
      k_collapse_cost<<<blocks_of(rd.second - rd.first, 256), 256, 0, s>>>(rd.first, rd.second, left, right, first,
                                                                         last, inner_box, leaf_box, leaf_max, cost,
                                                                         choice);
    AGS_CHECK(cudaGetLastError());
  }
  int h_err = 0;
  AGS_CHECK(cudaMemcpyAsync(roots.data(), d_roots, (size_t)E * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  AGS_CHECK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  AGS_CHECK(cudaStreamSynchronize(s));
  if (h_err) {
    set_error("clustering met an out-of-range node or position");
    return AGS_ERR_CUDA;
  }
  return AGS_OK;
}

}  // namespace ags
