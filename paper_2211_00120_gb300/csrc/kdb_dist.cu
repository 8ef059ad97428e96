// kdb_dist.cu -- the device steps of the sharded single-tree build.
//
// A single tree over points spread across several GPUs: the top levels are
// chosen across the shards, then every shard's points are sent to the GPU
// that owns their subtree, which builds it alone (kdb_build_subtree).  On the
// top levels each step is the paper's per-level step (Sec. 3): for every node
// the point of rank ss(lChild) in the node's order by (coordinate, original
// index) is its pivot (Observation 1), found by a radix select over the
// 64-bit key (coordinate key << 32 | original index) whose digit histograms
// are summed across the shards; then every point's tag moves to the child
// on its side of the pivot (Sec. 3.2).  The tag is the paper's one int32 per
// point: a node of the current level, or -1 once the point is pinned.
#include "kdb_launch.h"

namespace kdb {
namespace {

constexpr int kDistThreads = 256;

__device__ inline uint64_t dist_key64(const DistArgs& a, uint32_t i, int d) {
  const uint32_t bits = *reinterpret_cast<const uint32_t*>(a.pts + (uint64_t)i * (uint32_t)a.stride + 4u * d);
  return ((uint64_t)coord_key(bits, a.ctype) << 32) | (uint64_t)(a.index_base + i);
}

// The node (relative to the level's first node) of point i, or -1.
__device__ inline int dist_node(const DistArgs& a, uint32_t i) {
  const int32_t t = a.tags[i];
  if (t < (int32_t)a.first) return -1;
  const uint32_t u = (uint32_t)t - a.first;
  return u < a.nodes ? (int)u : -1;
}

// Digit histogram of every node's candidates: the points whose key agrees
// with the node's prefix in its top prefix_bits bits, by the next 8 bits.
__global__ void __launch_bounds__(kDistThreads) dist_hist_kernel(DistArgs a) {
  extern __shared__ uint32_t s_h[];
  const uint32_t H = a.nodes * 256u;
  for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) s_h[i] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int u = dist_node(a, i);
    if (u < 0) continue;
    const int d = a.node_dim[u];
    if (d >= a.k) {
      atomicOr(a.err, ERR_INTERNAL);
      continue;
    }
    const uint64_t key = dist_key64(a, i, d);
    if (a.prefix_bits > 0 && (key >> (64 - a.prefix_bits)) != a.prefix[u]) continue;
    atomicAdd(&s_h[u * 256u + ((uint32_t)(key >> (56 - a.prefix_bits)) & 255u)], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < H; i += blockDim.x)
    if (s_h[i]) atomicAdd(a.hist + i, s_h[i]);
}

// Smallest and largest coordinate key of every node's points in every
// dimension (the scene box at level 0, the tight boxes of the nodes).
__global__ void __launch_bounds__(kDistThreads) dist_box_kernel(DistArgs a) {
  extern __shared__ uint32_t s_b[];  // [nodes][2k]: min keys, then max keys
  const uint32_t B = a.nodes * 2u * (uint32_t)a.k;
  for (uint32_t i = threadIdx.x; i < B; i += blockDim.x) s_b[i] = (i / a.k) % 2u == 0 ? 0xFFFFFFFFu : 0u;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int u = dist_node(a, i);
    if (u < 0) continue;
    for (int d = 0; d < a.k; ++d) {
      const uint32_t key = (uint32_t)(dist_key64(a, i, d) >> 32);
      atomicMin(&s_b[u * 2u * a.k + d], key);
      atomicMax(&s_b[u * 2u * a.k + a.k + d], key);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < B; i += blockDim.x) {
    if ((i / a.k) % 2u == 0) atomicMin(a.box + i, s_b[i]);
    else atomicMax(a.box + i, s_b[i]);
  }
}

// Tag update of one top level (Sec. 3.2): below the node's pivot to child
// 2t+1, above it to 2t+2, the pivot itself pinned (tag -1, its position
// recorded for the node).
__global__ void __launch_bounds__(kDistThreads) dist_assign_kernel(DistArgs a) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int u = dist_node(a, i);
    if (u < 0) continue;
    const int d = a.node_dim[u];
    if (d >= a.k) {
      atomicOr(a.err, ERR_INTERNAL);
      continue;
    }
    const uint64_t key = dist_key64(a, i, d);
    const uint64_t piv = a.pivot[u];
    const int32_t t = a.tags[i];
    if (key < piv) a.tags[i] = 2 * t + 1;
    else if (key > piv) a.tags[i] = 2 * t + 2;
    else {
      a.tags[i] = -1;
      a.pinned[u] = (int64_t)i;
    }
  }
}

// Stable partition by destination (tag - first), in two steps: the items of
// each destination in every block's chunk, then (with each block's offsets
// per destination) the items themselves, written in chunk order.
__device__ inline void dist_chunk(const DistArgs& a, uint32_t* beg, uint32_t* end) {
  const uint64_t per = ((uint64_t)a.n + gridDim.x - 1) / gridDim.x;
  const uint64_t b = per * blockIdx.x, e = b + per;
  *beg = (uint32_t)(b < a.n ? b : a.n);
  *end = (uint32_t)(e < a.n ? e : a.n);
}

__global__ void __launch_bounds__(kDistThreads) dist_count_kernel(DistArgs a) {
  __shared__ uint32_t s_c[kDistMaxDest];
  for (int i = threadIdx.x; i < kDistMaxDest; i += blockDim.x) s_c[i] = 0;
  __syncthreads();
  uint32_t beg, end;
  dist_chunk(a, &beg, &end);
  for (uint32_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const int u = dist_node(a, i);
    if (u >= 0) atomicAdd(&s_c[u], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < a.nodes; i += blockDim.x) a.block_counts[blockIdx.x * a.nodes + i] = s_c[i];
}

__global__ void __launch_bounds__(kDistThreads) dist_scatter_kernel(DistArgs a) {
  constexpr int W = kDistThreads / 32;
  __shared__ uint32_t s_base[kDistMaxDest];       // the block's items of each destination so far
  __shared__ uint32_t s_wc[W][kDistMaxDest];      // per warp and destination: items, then offsets
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < kDistMaxDest; i += blockDim.x) s_base[i] = 0;
  uint32_t beg, end;
  dist_chunk(a, &beg, &end);
  const uint32_t* off = a.block_offsets + (uint64_t)blockIdx.x * a.nodes;
  const uint32_t words = (uint32_t)a.stride / 4u;
  for (uint32_t r0 = beg; r0 < end; r0 += blockDim.x) {
    for (int i = threadIdx.x; i < W * kDistMaxDest; i += blockDim.x) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const uint32_t i = r0 + threadIdx.x;
    const int u = i < end ? dist_node(a, i) : -1;
    const uint32_t peers = __match_any_sync(0xffffffffu, (uint32_t)u);
    const uint32_t rank = __popc(peers & lt);
    if (u >= 0 && (peers & lt) == 0) s_wc[warp][u] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < a.nodes) {  // destination u: offsets of the warps, base of the next round
      uint32_t run = s_base[threadIdx.x];
      for (int w = 0; w < W; ++w) {
        const uint32_t c = s_wc[w][threadIdx.x];
        s_wc[w][threadIdx.x] = run;
        run += c;
      }
      s_base[threadIdx.x] = run;
    }
    __syncthreads();
    if (u >= 0) {
      const uint64_t pos = (uint64_t)off[u] + s_wc[warp][u] + rank;
      if (pos >= a.n) {
        atomicOr(a.err, ERR_INTERNAL);
      } else {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(a.pts + (uint64_t)i * (uint32_t)a.stride);
        uint32_t* dst = reinterpret_cast<uint32_t*>(a.out_pts + pos * (uint32_t)a.stride);
        for (uint32_t q = 0; q < words; ++q) dst[q] = src[q];
        a.out_index[pos] = a.index_base + i;
      }
    }
    __syncthreads();
  }
}

// Memory-lean build (one GPU): the subtree rooted at node F(g) + rank, built
// in its own level order, goes to its nodes of the whole tree.  Local node q
// on the subtree's level lam is node F(g + lam) + (rank << lam) + (q - F(lam))
// of the whole tree (the level-order numbering of Sec. 2), so the nodes of
// one local level are one contiguous run.
__global__ void __launch_bounds__(kDistThreads) lean_place_kernel(LeanPlaceArgs a) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.m) return;
  const int lam = level_of(q);
  const uint64_t node = (uint64_t)full_nodes(a.g + lam) + ((uint64_t)a.rank << lam) + (q - full_nodes(lam));
  if (node >= a.total) {
    atomicOr(a.err, ERR_INTERNAL);
    return;
  }
  const uint32_t words = (uint32_t)a.stride / 4u;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(a.src + (uint64_t)q * (uint32_t)a.stride);
  uint32_t* dst = reinterpret_cast<uint32_t*>(a.dst + node * (uint32_t)a.stride);
  for (uint32_t w = 0; w < words; ++w) dst[w] = src[w];
}

// Memory-lean build: once a node's pivot has its coordinate key fixed, its
// index is one of the few points of the node with that key; they are
// gathered here instead of four more histogram passes over all points.
__global__ void __launch_bounds__(kDistThreads) lean_collect_kernel(DistArgs a, uint32_t cap, uint32_t* counts,
                                                                    uint32_t* out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int u = dist_node(a, i);
    if (u < 0) continue;
    const int d = a.node_dim[u];
    if (d >= a.k) {
      atomicOr(a.err, ERR_INTERNAL);
      continue;
    }
    if ((uint32_t)(dist_key64(a, i, d) >> 32) != (uint32_t)a.prefix[u]) continue;
    const uint32_t j = atomicAdd(&counts[u], 1u);
    if (j < cap) out[(uint64_t)u * cap + j] = a.index_base + i;
  }
}

__global__ void __launch_bounds__(kDistThreads) nan_check_kernel(const unsigned char* pts, uint32_t n, int k,
                                                                 int stride, uint32_t* err) {
  bool nan = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t* r = reinterpret_cast<const uint32_t*>(pts + (uint64_t)i * (uint32_t)stride);
    for (int d = 0; d < k; ++d)
      if ((r[d] & 0x7FFFFFFFu) > 0x7F800000u) nan = true;
  }
  if (__any_sync(0xffffffffu, nan) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_NAN);
}

uint32_t dist_grid(uint32_t n, int sms) {
  uint32_t g = (uint32_t)sms * 4u;
  const uint32_t need = (n + kDistThreads - 1) / kDistThreads;
  if (g > need) g = need;
  return g ? g : 1u;
}

}  // namespace

uint32_t dist_blocks(uint32_t n, int sms) { return dist_grid(n, sms); }

cudaError_t launch_dist_hist(const DistArgs& a, int sms, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const size_t smem = (size_t)a.nodes * 256 * sizeof(uint32_t);
  cudaError_t e = ensure_smem((const void*)dist_hist_kernel, smem);
  if (e != cudaSuccess) return e;
  dist_hist_kernel<<<dist_grid(a.n, sms), kDistThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dist_box(const DistArgs& a, int sms, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const size_t smem = (size_t)a.nodes * 2 * a.k * sizeof(uint32_t);
  dist_box_kernel<<<dist_grid(a.n, sms), kDistThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dist_assign(const DistArgs& a, int sms, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  dist_assign_kernel<<<dist_grid(a.n, sms), kDistThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dist_count(const DistArgs& a, uint32_t blocks, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  dist_count_kernel<<<blocks, kDistThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dist_scatter(const DistArgs& a, uint32_t blocks, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  dist_scatter_kernel<<<blocks, kDistThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_lean_place(const LeanPlaceArgs& a, cudaStream_t st) {
  if (a.m == 0) return cudaSuccess;
  lean_place_kernel<<<(a.m + kDistThreads - 1) / kDistThreads, kDistThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_lean_collect(const DistArgs& a, uint32_t cap, uint32_t* counts, uint32_t* out, int sms,
                                cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  lean_collect_kernel<<<dist_grid(a.n, sms), kDistThreads, 0, st>>>(a, cap, counts, out);
  return cudaGetLastError();
}

cudaError_t launch_nan_check(const unsigned char* pts, uint32_t n, int k, int stride, uint32_t* err, int sms,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  nan_check_kernel<<<dist_grid(n, sms), kDistThreads, 0, st>>>(pts, n, k, stride, err);
  return cudaGetLastError();
}

}  // namespace kdb
