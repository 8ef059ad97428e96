// kdb_local.cu -- finish small subtrees on chip.
//
// Once every subtree of a level holds at most 2^13 - 1 points, one thread
// block takes one subtree and runs all of its remaining levels in shared
// memory, writing only the final node -> point entries.
//
// Inside the block, each level still performs the paper's step: order every
// sub-segment by (tag, coordinate) (Sec. 3.1) and apply the tag update
// (Sec. 3.2).  The order is kept as k lists, one per dimension, each holding
// the block's points sorted by (sub-segment, rank in that dimension).  For a
// level with split dimension d, the list of d *is* the sorted order the tag
// update needs: in sub-segment t the point at rank ss(lChild) is pinned
// (Observation 1), lower ranks go left, higher ranks right.  Every list is
// then partitioned stably by that outcome, which leaves each child's points
// sorted by (child, rank) -- the next level's sort order -- without sorting
// again.  The lists are built once: the list of the parent's dimension comes
// in order (the items arrive sorted by it), the others are radix-sorted in
// shared memory.
#include "kdb_launch.h"

namespace kdb {
namespace {

constexpr int T = kLocalThreads;
constexpr int W = T / 32;
// nodes per level of a subtree finished by one warp (see the warp phase)
constexpr int kWarpTab = 1 << (kLocalLog - 1 - 5);
static_assert(W == 32, "the warp phase starts at the first depth with >= 32 subtrees");
// level-phase scratch: side + 3 node tables + dims + planes + warp tables
static_assert(kLocalCap + 3 * 2 * (kLocalCap / 2 + 8) + kLocalCap + 4 * kLocalCap +
                      W * 2 * kWarpTab * 2 <= 12 * kLocalCap,
              "level-phase scratch fits the sort area");

__device__ inline int widest_dim(const float* lo, const float* hi, int k) {
  int best = 0;
  float be = __fsub_rn(hi[0], lo[0]);
  for (int d = 1; d < k; ++d) {
    const float e = __fsub_rn(hi[d], lo[d]);
    if (e > be) {
      be = e;
      best = d;
    }
  }
  return best;
}

// Exclusive block scan of one value per thread (all T threads).
__device__ inline uint32_t scan_excl(uint32_t v, uint32_t* s_w, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t y = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    s_w[lane] = y;
  }
  __syncthreads();
  const uint32_t r = (w ? s_w[w - 1] : 0u) + x - v;
  if (total) *total = s_w[W - 1];
  __syncthreads();
  return r;
}

__device__ inline uint32_t block_min(uint32_t v, uint32_t* s_w) {
  v = __reduce_min_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t r = s_w[0];
  for (int i = 1; i < W; ++i) r = min(r, s_w[i]);
  __syncthreads();
  return r;
}

__device__ inline uint32_t block_max(uint32_t v, uint32_t* s_w) {
  v = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t r = s_w[0];
  for (int i = 1; i < W; ++i) r = max(r, s_w[i]);
  __syncthreads();
  return r;
}

// Stable LSD radix sort of m (key, index) pairs in shared memory, 8-bit
// digits, warp-match ranking.  Result in (ka, ia) if passes is even, else in
// (kb, ib); returns a pointer to the sorted index array.
__device__ uint16_t* smem_radix_sort(uint32_t* ka, uint16_t* ia, uint32_t* kb, uint16_t* ib,
                                     uint16_t* s_wh /* [256][W] */, uint32_t m, int passes,
                                     uint32_t* s_w) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  constexpr int PER = kLocalCap / T;  // items per thread (8)
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    for (int i = threadIdx.x; i < 256 * W; i += T) s_wh[i] = 0;
    __syncthreads();
    uint32_t key[PER];
    uint16_t rk[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const uint32_t i = (uint32_t)w * 32 * PER + r * 32 + lane;
      const bool ok = i < m;
      key[r] = ok ? ka[i] : 0u;
      const uint32_t d = ok ? (key[r] >> shift) & 255u : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = 0;
      if (ok) before = s_wh[d * W + w];
      __syncwarp();
      if (ok) {
        rk[r] = (uint16_t)(before + __popc(peers & lt));
        if ((peers & lt) == 0) s_wh[d * W + w] = (uint16_t)(before + __popc(peers));
      }
      __syncwarp();
    }
    __syncthreads();
    // digit-major exclusive scan of the 256 x W counters
    constexpr int CPT = 256 * W / T;  // counters per thread (8)
    uint32_t c[CPT], sum = 0;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      c[q] = s_wh[threadIdx.x * CPT + q];
      sum += c[q];
    }
    uint32_t run = scan_excl(sum, s_w, nullptr);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      s_wh[threadIdx.x * CPT + q] = (uint16_t)run;
      run += c[q];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const uint32_t i = (uint32_t)w * 32 * PER + r * 32 + lane;
      if (i < m) {
        const uint32_t d = (key[r] >> shift) & 255u;
        const uint32_t pos = s_wh[d * W + w] + rk[r];
        kb[pos] = key[r];
        ib[pos] = ia[i];
      }
    }
    __syncthreads();
    uint32_t* kt = ka;
    ka = kb;
    kb = kt;
    uint16_t* it = ia;
    ia = ib;
    ib = it;
  }
  return ia;
}

__global__ void __launch_bounds__(T, 1) local_finish_kernel(LocalArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t s_w[W];
  __shared__ float s_box[2 * kMaxK];
  __shared__ int s_list_of[kMaxK + 1];  // physical list slot of each dimension, + spare
  __shared__ uint32_t s_bad;
  if (*reinterpret_cast<volatile uint32_t*>(a.err)) return;
  const int k = a.k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t* s_orig = reinterpret_cast<uint32_t*>(sm);                      // kLocalCap
  uint16_t* s_lists = reinterpret_cast<uint16_t*>(s_orig + kLocalCap);     // (k+1) * cap
  unsigned char* s_area = reinterpret_cast<unsigned char*>(s_lists + (size_t)(k + 1) * kLocalCap);
  // sort phase view of the scratch area
  uint32_t* s_ka = reinterpret_cast<uint32_t*>(s_area);
  uint32_t* s_kb = s_ka + kLocalCap;
  uint16_t* s_ia = reinterpret_cast<uint16_t*>(s_kb + kLocalCap);
  uint16_t* s_ib = s_ia + kLocalCap;
  // level phase view of the scratch area
  uint8_t* s_side = s_area;                                                  // cap
  uint16_t* s_tstart = reinterpret_cast<uint16_t*>(s_area + kLocalCap);      // cap/2 + 1
  uint16_t* s_tpr = s_tstart + kLocalCap / 2 + 8;                            // cap/2
  uint16_t* s_tpl = s_tpr + kLocalCap / 2 + 8;                               // cap/2
  uint8_t* s_ldim = reinterpret_cast<uint8_t*>(s_tpl + kLocalCap / 2 + 8);   // cap
  float* s_lplane = reinterpret_cast<float*>(s_ldim + kLocalCap);            // cap

  const LocalWork wk = a.work[blockIdx.x];
  const LocalSet ls = a.lsets[wk.set];
  const Tree tree = make_tree(ls.n);
  const int l0 = ls.l0;
  const uint32_t s0 = full_nodes(l0) + wk.s_rel;
  const LevelLayout y0 = LevelLayout::make(tree, l0);
  const uint32_t start0 = y0.seg_start(wk.s_rel);
  const uint32_t m = y0.seg_start(wk.s_rel + 1) - start0;
  if (m == 0) return;
  if (m > (uint32_t)kLocalMax) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_INTERNAL);
    return;
  }
  if (threadIdx.x == 0) s_bad = 0;
  // entries (k <= 3) carry every rank; otherwise ranks are gathered
  const uint4* ents = nullptr;
  if (a.ents_local) ents = l0 > 0 ? a.ents_local + ls.off + start0 : a.rows + ls.off;
  for (uint32_t i = threadIdx.x; i < m; i += T)
    s_orig[i] = ents ? ents[i].w : (l0 > 0 ? a.vals_local[ls.off + start0 + i] : ls.off + i);
  if (threadIdx.x <= (unsigned)k) s_list_of[threadIdx.x] = threadIdx.x;
  __syncthreads();

  // dimension the items arrive sorted by: the parent's split dimension
  int dpar = -1;
  if (l0 > 0) dpar = a.mode == 0 ? (l0 - 1) % k : a.dims[ls.off + (s0 - 1) / 2];
  // the spare list slot holds the radix counters while the lists are built
  uint16_t* s_wh = s_lists + (size_t)k * kLocalCap;
  if (ents) {
    // Lists ordered by (key_d, original index).  The items arrive ordered so
    // in the parent's split dimension (on a set's level 0: by index).  For
    // the other dimensions the items are put in index order once, then
    // sorted stably by key from that order.
    int todo[kMaxK];
    int nt = 0;
    for (int d = 0; d < k; ++d)
      if (d != dpar) todo[nt++] = d;
    if (dpar >= 0) {
      uint16_t* list = s_lists + (size_t)dpar * kLocalCap;
      for (uint32_t i = threadIdx.x; i < m; i += T) list[i] = (uint16_t)i;
    }
    if (nt > 0) {
      uint16_t* ord = s_lists + (size_t)todo[nt - 1] * kLocalCap;  // index order
      if (l0 > 0) {
        uint32_t lo = 0xFFFFFFFFu, hi = 0;
        for (uint32_t i = threadIdx.x; i < m; i += T) {
          lo = min(lo, s_orig[i]);
          hi = max(hi, s_orig[i]);
        }
        lo = block_min(lo, s_w);
        hi = block_max(hi, s_w);
        for (uint32_t i = threadIdx.x; i < m; i += T) {
          s_ka[i] = s_orig[i] - lo;
          s_ia[i] = (uint16_t)i;
        }
        __syncthreads();
        const int passes = (bits_for((uint64_t)(hi - lo) + 1) + 7) / 8;
        const uint16_t* sorted = smem_radix_sort(s_ka, s_ia, s_kb, s_ib, s_wh, m, passes, s_w);
        for (uint32_t i = threadIdx.x; i < m; i += T) ord[i] = sorted[i];
      } else {
        for (uint32_t i = threadIdx.x; i < m; i += T) ord[i] = (uint16_t)i;
      }
      __syncthreads();
      for (int q = 0; q < nt; ++q) {
        const int d = todo[q];
        uint32_t lo = 0xFFFFFFFFu, hi = 0;
        for (uint32_t i = threadIdx.x; i < m; i += T) {
          const uint16_t it = ord[i];
          const uint4 e = ents[it];
          const uint32_t key = d == 0 ? e.x : (d == 1 ? e.y : e.z);
          s_ka[i] = key;
          s_ia[i] = it;
          lo = min(lo, key);
          hi = max(hi, key);
        }
        lo = block_min(lo, s_w);
        hi = block_max(hi, s_w);
        for (uint32_t i = threadIdx.x; i < m; i += T) s_ka[i] -= lo;
        __syncthreads();
        const int passes = (bits_for((uint64_t)(hi - lo) + 1) + 7) / 8;
        const uint16_t* sorted = smem_radix_sort(s_ka, s_ia, s_kb, s_ib, s_wh, m, passes, s_w);
        uint16_t* list = s_lists + (size_t)d * kLocalCap;
        for (uint32_t i = threadIdx.x; i < m; i += T) list[i] = sorted[i];
        __syncthreads();
      }
    }
  } else {
  for (int d = 0; d < k; ++d) {
    uint16_t* list = s_lists + (size_t)d * kLocalCap;
    if (d == dpar) {
      for (uint32_t i = threadIdx.x; i < m; i += T) list[i] = (uint16_t)i;
      continue;
    }
    const uint32_t* rank_d = a.ranks + (size_t)d * a.total;
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    for (uint32_t i = threadIdx.x; i < kLocalCap; i += T) {
      uint32_t r = 0xFFFFFFFFu;
      if (i < m) {
        const uint32_t o = s_orig[i];
        if (o < a.total) r = rank_d[o];
        else s_bad = 1;
        lo = min(lo, r);
        hi = max(hi, r);
      }
      s_ka[i] = r;
      s_ia[i] = (uint16_t)i;
    }
    lo = block_min(lo, s_w);
    hi = block_max(hi, s_w);
    for (uint32_t i = threadIdx.x; i < m; i += T) s_ka[i] -= lo;
    __syncthreads();
    const int passes = (bits_for((uint64_t)(hi - lo) + 1) + 7) / 8;
    const uint16_t* sorted = smem_radix_sort(s_ka, s_ia, s_kb, s_ib, s_wh, m, passes, s_w);
    for (uint32_t i = threadIdx.x; i < m; i += T) list[i] = sorted[i];
    __syncthreads();
  }
  }

  // domain of the subtree root (widest mode)
  if (a.mode == 1 && threadIdx.x == 0) {
    if (l0 == 0) {
      for (int d = 0; d < k; ++d) {
        s_box[d] = __uint_as_float(key_to_float_bits(a.bbox[wk.set * 2 * k + d]));
        s_box[kMaxK + d] = __uint_as_float(key_to_float_bits(a.bbox[wk.set * 2 * k + k + d]));
      }
      const int d0 = widest_dim(s_box, s_box + kMaxK, k);
      a.dims[ls.off + s0] = (uint8_t)d0;
      s_ldim[0] = (uint8_t)d0;
    } else {
      const float* b = a.boxes_local + ((size_t)ls.lbox0 + wk.s_rel) * 2 * k;
      for (int d = 0; d < k; ++d) {
        s_box[d] = b[d];
        s_box[kMaxK + d] = b[k + d];
      }
      s_ldim[0] = a.dims[ls.off + s0];
    }
  }
  __syncthreads();

  uint32_t mj = m;  // live items at this depth
  for (int j = 0;; ++j) {
    const int L = l0 + j;  // level of this depth in the set's tree
    if (L > tree.L - 1 || mj == 0) break;
    const LevelLayout yj = LevelLayout::make(tree, L);
    const uint32_t first = (((s0 + 1) << j) - 1) - full_nodes(L);  // subtree rel index of t = 0
    const uint32_t nodes = 1u << j;
    const uint32_t base = yj.seg_start(first);
    // nodes of this depth that exist (only the lowest level can be partial)
    uint32_t nn = nodes;
    if (L == tree.L - 1) {
      const uint32_t c0 = ((s0 + 1) << j) - 1;
      nn = c0 >= tree.n ? 0 : min(nodes, tree.n - c0);
    }
    if (nodes >= (uint32_t)W) {
      // From here on every subtree of this depth is finished by one warp,
      // independently of the others.  Within its subtree a warp keeps each
      // node's points in the node's in-order range: the left child takes
      // [start, start + pr), the pivot's slot stays empty, the right child
      // takes (start + pr, start + size).  Ranges of different warps never
      // overlap, so warps need no block barrier and each keeps its own list
      // rotation.
      // a warp's subtree has at most 2^(kLocalLog-5) - 1 points, so at most
      // kWarpTab nodes on any of its levels; two tables per warp
      const uint32_t c0 = ((s0 + 1) << j) - 1;
      uint16_t* tabs = reinterpret_cast<uint16_t*>(s_lplane + kLocalCap) + (size_t)warp * 2 * kWarpTab;
      for (uint32_t t = warp; t < nn; t += W) {
        int slot[kMaxK + 1];
        for (int q = 0; q <= k; ++q) slot[q] = s_list_of[q];
        uint16_t* ta = tabs;
        uint16_t* tb2 = tabs + kWarpTab;
        const uint32_t root = c0 + t;
        if (lane == 0) ta[0] = (uint16_t)(yj.seg_start(first + t) - base);
        __syncwarp();
        for (int i = 0;; ++i) {
          const int Li = L + i;
          if (Li > tree.L - 1) break;
          const uint32_t cf = ((root + 1) << i) - 1;  // first node of sub-depth i
          if (cf >= tree.n) break;
          const uint32_t cnt = min(1u << i, tree.n - cf);
          const bool lowest = Li == tree.L - 1;
          const uint32_t jj = j + i;                    // depth below s0
          const uint32_t loc0 = (1u << jj) - 1 + (t << i);  // local index of node cf
          const bool coop = cnt <= 8;  // few nodes: the warp shares each node's items
          // pins, sides, widest dimensions
          for (uint32_t u = coop ? 0u : (uint32_t)lane; u < cnt; u += coop ? 1u : 32u) {
            const uint32_t node = cf + u;
            const uint32_t st = ta[u];
            const uint32_t sz = subtree_size(tree, node);
            const uint32_t pr = subtree_size(tree, 2 * node + 1);
            int d = Li % k;
            if (a.mode == 1) {
              float lo[kMaxK], hi[kMaxK];
              for (int dd = 0; dd < k; ++dd) {
                lo[dd] = s_box[dd];
                hi[dd] = s_box[kMaxK + dd];
              }
              const uint32_t tt = (t << i) + u;  // index among depth-jj nodes of s0
              for (uint32_t e = 0; e < jj; ++e) {
                const uint32_t la = (1u << e) - 1 + (tt >> (jj - e));
                const int da = s_ldim[la];
                const float xv = s_lplane[la];
                if (((tt >> (jj - 1 - e)) & 1u) == 0) hi[da] = xv; else lo[da] = xv;
              }
              d = widest_dim(lo, hi, k);
            }
            const uint16_t* list = s_lists + (size_t)slot[d] * kLocalCap;
            if (!coop || lane == 0) {
              const uint32_t o = s_orig[list[st + pr]];
              a.perm[ls.off + node] = o;
              if (a.mode == 1) {
                s_ldim[loc0 + u] = (uint8_t)d;
                s_lplane[loc0 + u] = coord_of(a.pts, o, a.stride, d);
                a.dims[ls.off + node] = (uint8_t)d;
              }
            }
            for (uint32_t q = coop ? (uint32_t)lane : 0u; q < sz; q += coop ? 32u : 1u)
              s_side[list[st + q]] = q < pr ? 0 : (q == pr ? 2 : 1);
          }
          __syncwarp();
          if (lowest) break;
          const int depth_left = tree.L - 1 - (Li + 1);
          for (int dd = 0; dd < k; ++dd) {
            if (a.mode == 0) {
              bool need = false;
              for (int q = 0; q <= depth_left && !need; ++q) need = ((Li + 1 + q) % k) == dd;
              if (!need) continue;
            }
            const uint16_t* src = s_lists + (size_t)slot[dd] * kLocalCap;
            uint16_t* dst = s_lists + (size_t)slot[k] * kLocalCap;
            for (uint32_t u = coop ? 0u : (uint32_t)lane; u < cnt; u += coop ? 1u : 32u) {
              const uint32_t node = cf + u;
              const uint32_t st = ta[u];
              const uint32_t sz = subtree_size(tree, node);
              const uint32_t pr = subtree_size(tree, 2 * node + 1);
              uint32_t cl = 0, cr = 0;
              if (coop) {
                for (uint32_t q0 = 0; q0 < sz; q0 += 32) {
                  const uint32_t q = q0 + lane;
                  uint16_t it = 0;
                  uint8_t sd = 3;
                  if (q < sz) {
                    it = src[st + q];
                    sd = s_side[it];
                  }
                  const uint32_t bl = __ballot_sync(0xffffffffu, sd == 0);
                  const uint32_t br = __ballot_sync(0xffffffffu, sd == 1);
                  if (sd == 0) dst[st + cl + __popc(bl & lt)] = it;
                  if (sd == 1) dst[st + pr + 1 + cr + __popc(br & lt)] = it;
                  cl += __popc(bl);
                  cr += __popc(br);
                }
              } else {
                for (uint32_t q = 0; q < sz; ++q) {
                  const uint16_t it = src[st + q];
                  const uint8_t sd = s_side[it];
                  if (sd == 0) dst[st + cl++] = it;
                  else if (sd == 1) dst[st + pr + 1 + cr++] = it;
                }
              }
            }
            __syncwarp();
            const int t2 = slot[dd];
            slot[dd] = slot[k];
            slot[k] = t2;
          }
          // children's ranges: left starts where the node starts, right after the pivot
          for (uint32_t u = lane; u < cnt; u += 32) {
            const uint32_t st = ta[u];
            const uint32_t pr = subtree_size(tree, 2 * (cf + u) + 1);
            tb2[2 * u] = (uint16_t)st;
            tb2[2 * u + 1] = (uint16_t)(st + pr + 1);
          }
          __syncwarp();
          uint16_t* tt2 = ta;
          ta = tb2;
          tb2 = tt2;
        }
      }
      break;
    }
    // per node: segment start, pivot rank, lefts before it
    for (uint32_t t = threadIdx.x; t < nn; t += T) {
      s_tstart[t] = (uint16_t)(yj.seg_start(first + t) - base);
      s_tpr[t] = (uint16_t)(yj.h >= 1 ? yj.left_size(first + t) : 0u);
    }
    if (threadIdx.x == 0) s_tstart[nn] = (uint16_t)mj;
    __syncthreads();
    {
      // exclusive scan of the pivot ranks over the nodes (<= 4 per thread)
      const uint32_t per = (nn + T - 1) / T;
      const uint32_t t0 = threadIdx.x * per;
      uint32_t v[4] = {0, 0, 0, 0}, sum = 0;
      for (uint32_t q = 0; q < per && q < 4; ++q)
        if (t0 + q < nn) {
          v[q] = s_tpr[t0 + q];
          sum += v[q];
        }
      uint32_t run = scan_excl(sum, s_w, nullptr);
      for (uint32_t q = 0; q < per && q < 4; ++q)
        if (t0 + q < nn) {
          s_tpl[t0 + q] = (uint16_t)run;
          run += v[q];
        }
    }
    // split dimension of every node of this depth (widest: clipped domain)
    if (a.mode == 1 && j > 0) {
      for (uint32_t t = threadIdx.x; t < nn; t += T) {
        float lo[kMaxK], hi[kMaxK];
        for (int d = 0; d < k; ++d) {
          lo[d] = s_box[d];
          hi[d] = s_box[kMaxK + d];
        }
        for (int i = 0; i < j; ++i) {
          const uint32_t ti = t >> (j - i);
          const uint32_t loc = (1u << i) - 1 + ti;
          const int da = s_ldim[loc];
          const float x = s_lplane[loc];
          if (((t >> (j - 1 - i)) & 1u) == 0) hi[da] = x; else lo[da] = x;
        }
        const int dd = widest_dim(lo, hi, k);
        s_ldim[(1u << j) - 1 + t] = (uint8_t)dd;
        a.dims[ls.off + ((s0 + 1) << j) - 1 + t] = (uint8_t)dd;
      }
    }
    __syncthreads();
    const int drr = L % k;
    // pin the pivots; mark every item left / pivot / right
    for (uint32_t t = threadIdx.x; t < nn; t += T) {
      const int d = a.mode == 0 ? drr : s_ldim[(1u << j) - 1 + t];
      const uint16_t* list = s_lists + (size_t)s_list_of[d] * kLocalCap;
      const uint32_t it = list[s_tstart[t] + s_tpr[t]];
      const uint32_t o = s_orig[it];
      a.perm[ls.off + ((s0 + 1) << j) - 1 + t] = o;
      if (a.mode == 1) s_lplane[(1u << j) - 1 + t] = coord_of(a.pts, o, a.stride, d);
    }
    {
      const uint32_t per = (mj + T - 1) / T;
      const uint32_t p0 = threadIdx.x * per, p1 = min(p0 + per, mj);
      uint32_t t = 0;
      if (p0 < p1) {
        uint32_t lo = 0, hi = nn;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (s_tstart[mid] <= p0) lo = mid; else hi = mid;
        }
        t = lo;
      }
      for (uint32_t p = p0; p < p1; ++p) {
        while (t + 1 < nn && s_tstart[t + 1] <= p) ++t;
        const int d = a.mode == 0 ? drr : s_ldim[(1u << j) - 1 + t];
        const uint16_t* list = s_lists + (size_t)s_list_of[d] * kLocalCap;
        const uint32_t q = p - s_tstart[t], pr = s_tpr[t];
        s_side[list[p]] = q < pr ? 0 : (q == pr ? 2 : 1);
      }
    }
    __syncthreads();
    if (L == tree.L - 1) break;  // lowest level: every item was pinned
    // stable partition of every list still needed into the next depth's order
    const uint32_t mn = mj - nn;
    const int depth_left = tree.L - 1 - (L + 1);  // levels after the next one
    for (int d = 0; d < k; ++d) {
      if (a.mode == 0) {
        bool need = false;
        for (int jj = 0; jj <= depth_left && !need; ++jj) need = ((L + 1 + jj) % k) == d;
        if (!need) continue;
      }
      const int src_slot = s_list_of[d], dst_slot = s_list_of[k];
      const uint16_t* src = s_lists + (size_t)src_slot * kLocalCap;
      uint16_t* dst = s_lists + (size_t)dst_slot * kLocalCap;
      const uint32_t per = (mj + T - 1) / T;
      const uint32_t p0 = threadIdx.x * per, p1 = min(p0 + per, mj);
      uint32_t cnt = 0;  // lefts in the low half, rights in the high half
      for (uint32_t p = p0; p < p1; ++p) {
        const uint8_t sd = s_side[src[p]];
        cnt += sd == 0 ? 1u : (sd == 1 ? 0x10000u : 0u);
      }
      uint32_t run = scan_excl(cnt, s_w, nullptr);
      uint32_t gl = run & 0xFFFFu, gr = run >> 16;
      uint32_t t = 0;
      if (p0 < p1) {
        uint32_t lo = 0, hi = nn;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (s_tstart[mid] <= p0) lo = mid; else hi = mid;
        }
        t = lo;
      }
      for (uint32_t p = p0; p < p1; ++p) {
        while (t + 1 < nn && s_tstart[t + 1] <= p) ++t;
        const uint16_t it = src[p];
        const uint8_t sd = s_side[it];
        if (sd == 2) continue;
        const uint32_t ts = s_tstart[t], pr = s_tpr[t], pl = s_tpl[t];
        uint32_t np;
        if (sd == 0) {
          np = ts - t + (gl - pl);
          ++gl;
        } else {
          np = ts - t + pr + (gr - (ts - t - pl));
          ++gr;
        }
        if (np < mn) dst[np] = it;
        else s_bad = 1;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_list_of[d] = dst_slot;
        s_list_of[k] = src_slot;
      }
      __syncthreads();
    }
    mj = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_bad) atomicOr(a.err, ERR_INTERNAL);
}

}  // namespace

size_t local_smem_bytes(int k) {
  return (size_t)kLocalCap * 4 + (size_t)(k + 1) * kLocalCap * 2 + (size_t)kLocalCap * 12;
}

cudaError_t launch_local_finish(const LocalArgs& a, cudaStream_t st) {
  if (a.nwork == 0) return cudaSuccess;
  const size_t smem = local_smem_bytes(a.k);
  cudaError_t e = cudaFuncSetAttribute(local_finish_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  local_finish_kernel<<<a.nwork, T, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace kdb
