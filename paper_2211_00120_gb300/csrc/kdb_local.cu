// kdb_local.cu -- finish small subtrees on chip.
//
// Once every subtree of a level holds at most 2^13 - 1 points, one thread
// block takes one subtree and runs all of its remaining levels in shared
// memory, writing only the final node -> point entries.
//
// Inside the block, each level still performs the paper's step: order every
// sub-segment by (tag, coordinate) (Sec. 3.1) and apply the tag update
// (Sec. 3.2).  The order is kept as k lists of local ids, one per dimension,
// each sorted by (sub-segment, key_d, original index).  For a level with split
// dimension d, the list of d *is* the sorted order the tag update needs: in
// sub-segment t the point at rank ss(lChild) is pinned (Observation 1), lower
// ranks go left, higher ranks right.  One pass over that list writes, per
// point, its side and the closed-form start of its run on the next level (the
// sub-segment sizes of Sec. 4); every list is then partitioned stably by side
// with warp ballots, which leaves each child's points sorted by (child, key,
// index) -- the next level's sort order -- without sorting again.  Once a
// depth has at least 32 sub-segments, each warp finishes its own subtrees
// without block barriers.
//
// The lists arrive from the global passes already in order (as original
// indices); a set small enough to start here builds them from its entries by
// radix sorts in shared memory.
#include "kdb_launch.h"

namespace kdb {
namespace {

constexpr int T = kLocalThreads;
constexpr int W = T / 32;
static_assert(W == 32, "the warp phase starts at the first depth with >= 32 subtrees");
// scratch area (12 bytes per item): the setup's sort buffers (4 + 4 + 2 + 2)
// or hash table (2 slots per item of 4 + 2 bytes); the levels' info words,
// split dimensions and planes (2 + 1 + 4)
static_assert(2 * kLocalCap * 4 + 2 * kLocalCap * 2 <= 12 * kLocalCap, "hash table fits");
static_assert(kLocalCap * (2 + 1 + 4) <= 12 * kLocalCap, "level scratch fits");
static_assert(kLocalCap <= (1 << 14), "info words hold 14-bit offsets");

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

// Slot of list d among the k + 1 list buffers, packed 4 bits per dimension
// (the last one is the spare that receives a partition).
__device__ inline int slot_of(uint32_t slots, int d) { return (int)((slots >> (4 * d)) & 15u); }
__device__ inline uint32_t swap_slots(uint32_t slots, int d, int k) {
  const uint32_t a = (slots >> (4 * d)) & 15u, b = (slots >> (4 * k)) & 15u;
  slots &= ~((15u << (4 * d)) | (15u << (4 * k)));
  return slots | (b << (4 * d)) | (a << (4 * k));
}

// The block's subtree on one level of the set's tree, in block-local terms:
// segment u = the block's u-th subtree on that level, positions counted from
// the block's first item on that level.  Same closed forms as the set's
// layout (Sec. 4.1, 4.2) with the lowest-level nodes that fall inside the
// block's subtree; every value is below 2^13, so all of it is 32-bit.
struct Local {
  uint32_t h;        // levels below this one
  uint32_t thin;     // 2^h - 1: a subtree without lowest-level nodes
  uint32_t full;     // 2^(h+1) - 1
  uint32_t mb;       // lowest-level nodes inside the block's subtree
  uint32_t w;        // 2^(h-1): lowest-level width of a left child (h >= 1)
};

__device__ inline Local make_local(const Tree& tree, int L, uint32_t tfirst, uint32_t nodes) {
  Local y;
  y.h = (uint32_t)(tree.L - L - 1);
  y.thin = (1u << y.h) - 1u;
  y.full = 2u * y.thin + 1u;
  const uint64_t lo = (uint64_t)tfirst << y.h;  // first lowest-level slot of the block
  const uint64_t room = (uint64_t)nodes << y.h;
  y.mb = tree.m > lo ? (uint32_t)min((uint64_t)tree.m - lo, room) : 0u;
  y.w = y.h >= 1 ? 1u << (y.h - 1) : 0u;
  return y;
}
__device__ inline uint32_t l_start(const Local& y, uint32_t u) { return u * y.thin + min(u << y.h, y.mb); }
__device__ inline uint32_t l_left(const Local& y, uint32_t u) {  // h >= 1
  const uint32_t lowest = (2u * u) << (y.h - 1);
  const uint32_t low = lowest >= y.mb ? 0u : min(y.mb - lowest, y.w);
  return (y.w - 1u) + low;
}
__device__ inline uint32_t l_left_before(const Local& y, uint32_t u) {  // h >= 1
  const uint32_t fb = y.mb >> y.h;
  uint32_t low = min(u, fb) * y.w;
  if (u > fb) low += min(y.mb - fb * (2u * y.w), y.w);
  return u * (y.w - 1u) + low;
}

// Segments [uf, uf + cnt) of one level handled by one thread group.
struct Range {
  Local y;
  uint32_t uf;       // first segment
  uint32_t p0, p1;   // positions of the range's items
  uint32_t lb0;      // lefts before uf
  uint32_t nb;       // position of the range's first item on the next level
};

__device__ inline Range make_range(const Local& y, uint32_t uf, uint32_t cnt) {
  Range r;
  r.y = y;
  r.uf = uf;
  r.p0 = l_start(y, uf);
  r.p1 = l_start(y, uf + cnt);
  r.lb0 = y.h >= 1 ? l_left_before(y, uf) : 0u;
  // the next level holds every item of this level but the pinned ones, in
  // segment order: items before the range's first child = items before uf
  // minus the uf pivots above them
  r.nb = r.p0 - uf;
  return r;
}

// kMode: the split rule (0 round robin, 1 clipped domain, 2 tight box), a
// template argument so that each rule's kernel carries only its own code.
template <int kMode>
__global__ void __launch_bounds__(T, 1) local_finish_kernel(LocalArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t s_w[W];
  __shared__ float s_box[2 * kMaxK];
  __shared__ uint32_t s_bad;
  if (*reinterpret_cast<volatile uint32_t*>(a.err)) return;
  const int k = a.k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t* s_orig = reinterpret_cast<uint32_t*>(sm);                      // kLocalCap
  uint16_t* s_lists = reinterpret_cast<uint16_t*>(s_orig + kLocalCap);     // (k+1) * cap
  unsigned char* s_area = reinterpret_cast<unsigned char*>(s_lists + (size_t)(k + 1) * kLocalCap);
  // setup view of the scratch area: radix sort buffers, or the hash table
  uint32_t* s_ka = reinterpret_cast<uint32_t*>(s_area);
  uint32_t* s_kb = s_ka + kLocalCap;
  uint16_t* s_ia = reinterpret_cast<uint16_t*>(s_kb + kLocalCap);
  uint16_t* s_ib = s_ia + kLocalCap;
  uint32_t* s_hkey = reinterpret_cast<uint32_t*>(s_area);                  // 2 * cap
  uint16_t* s_hval = reinterpret_cast<uint16_t*>(s_hkey + 2 * kLocalCap);  // 2 * cap
  // level view of the scratch area
  uint16_t* s_info = reinterpret_cast<uint16_t*>(s_area);                  // cap
  uint8_t* s_ldim = reinterpret_cast<uint8_t*>(s_info + kLocalCap);        // cap
  float* s_lplane = reinterpret_cast<float*>(s_ldim + kLocalCap);          // cap

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
  __syncthreads();

  // ---- the k lists: local ids 0..m-1 ordered by (key_d, original index)
  int dpar = -1;  // dimension the items arrive sorted by (the parent's split)
  if (l0 > 0) dpar = kMode == 0 ? (l0 - 1) % k : a.dims[ls.off + (s0 - 1) / 2];
  uint16_t* s_wh = s_lists + (size_t)k * kLocalCap;  // radix counters (spare list slot)
  if (a.lorig && l0 > 0) {
    // The global passes hand over every list of the subtree as original
    // indices, already in order.  Local id = position in list 0; the other
    // lists are translated through a hash table original index -> local id.
    const uint32_t* lo0 = a.lorig + ls.off + start0;
    const uint4* le0 = a.lents ? a.lents + ls.off + start0 : nullptr;  // list 0 as entries
    constexpr uint32_t HM = 2 * kLocalCap - 1;
    for (uint32_t i = threadIdx.x; i < 2 * kLocalCap; i += T) s_hkey[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += T) {
      uint32_t o = le0 ? le0[i].w : lo0[i];
      if (o >= a.total) {
        s_bad = 1;
        o = 0;
      }
      s_orig[i] = o;
      s_lists[i] = (uint16_t)i;
      uint32_t h = (o * 0x9E3779B1u) >> (32 - (kLocalLog + 1));
      bool done = false;
      for (uint32_t probe = 0; probe <= HM && !done; ++probe) {
        const uint32_t prev = atomicCAS(&s_hkey[h], 0xFFFFFFFFu, o);
        if (prev == 0xFFFFFFFFu) {
          s_hval[h] = (uint16_t)i;
          done = true;
        } else if (prev == o) {
          break;  // an original index twice: corrupt input lists
        }
        h = (h + 1) & HM;
      }
      if (!done) s_bad = 1;
    }
    __syncthreads();
    for (int d = 1; d < k; ++d) {
      const uint32_t* lod = a.lorig + (size_t)d * a.total + ls.off + start0;
      uint16_t* list = s_lists + (size_t)d * kLocalCap;
      for (uint32_t i = threadIdx.x; i < m; i += T) {
        const uint32_t o = lod[i];
        uint32_t h = (o * 0x9E3779B1u) >> (32 - (kLocalLog + 1));
        uint32_t id = 0xFFFFFFFFu;
        for (uint32_t probe = 0; probe <= HM; ++probe) {
          const uint32_t key = s_hkey[h];
          if (key == o) {
            id = s_hval[h];
            break;
          }
          if (key == 0xFFFFFFFFu) break;
          h = (h + 1) & HM;
        }
        if (id >= m) {
          s_bad = 1;
          id = 0;
        }
        list[i] = (uint16_t)id;
      }
    }
    __syncthreads();
  } else if (a.rows) {
    // a set finished locally from its level 0: entries in input order carry
    // the keys; every list is a stable key sort from index order
    const uint4* ents = a.rows + ls.off;
    for (uint32_t i = threadIdx.x; i < m; i += T) {
      const uint32_t o = ents[i].w;
      if (o >= a.total) s_bad = 1;
      s_orig[i] = o < a.total ? o : 0u;
    }
    for (int d = 0; d < k; ++d) {
      uint32_t lo = 0xFFFFFFFFu, hi = 0;
      for (uint32_t i = threadIdx.x; i < m; i += T) {
        const uint4 e = ents[i];
        const uint32_t key = d == 0 ? e.x : (d == 1 ? e.y : e.z);
        s_ka[i] = key;
        s_ia[i] = (uint16_t)i;
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
  } else {
    // rank arrays (k > 3): the items arrive in the parent's order
    for (uint32_t i = threadIdx.x; i < m; i += T)
      s_orig[i] = l0 > 0 ? a.vals_local[ls.off + start0 + i] : ls.off + i;
    __syncthreads();
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

  // every list slot holds a local id below m at every position below m, the
  // spare slot included (it served as radix counters above): list reads stay
  // in range even if a consistency check has failed
  {
    uint16_t* spare = s_lists + (size_t)k * kLocalCap;
    for (uint32_t i = threadIdx.x; i < m; i += T) spare[i] = 0;
  }
  __syncthreads();

  // domain of the subtree root (widest mode)
  if (kMode == 1 && threadIdx.x == 0) {
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

  constexpr bool widest = kMode == 1;  // widest side of the clipped domain (Sec. 6)
  constexpr bool tight = kMode == 2;   // widest side of the subtree's own box
  constexpr bool bydim = widest || tight;
  // records written directly at their nodes: the entry of each local id
  const uint4* ent_of = nullptr;
  if (a.pts_out) ent_of = l0 > 0 ? a.lents + ls.off + start0 : a.rows + ls.off;
  // keys of each local id (tight-box rule: list 0 is handed over as entries)
  const uint4* key_of = nullptr;
  if (tight) key_of = l0 > 0 ? a.lents + ls.off + start0 : a.rows + ls.off;
  if (tight && !key_of) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_INTERNAL);
    return;
  }
  // split dimension of node tl (index among the block's nodes at depth jj):
  // widest side of its domain, the root's domain clipped by the planes of
  // its ancestors inside the block (Sec. 6)
  auto node_dim = [&](uint32_t jj, uint32_t tl) -> int {
    float lo[kMaxK], hi[kMaxK];
    for (int d = 0; d < k; ++d) {
      lo[d] = s_box[d];
      hi[d] = s_box[kMaxK + d];
    }
    for (uint32_t e = 0; e < jj; ++e) {
      const uint32_t la = (1u << e) - 1 + (tl >> (jj - e));
      const int da = s_ldim[la];
      const float xv = s_lplane[la];
      if (((tl >> (jj - 1 - e)) & 1u) == 0) hi[da] = xv; else lo[da] = xv;
    }
    return widest_dim(lo, hi, k);
  };
  // split dimension under the tight-box rule of the node whose items sit at
  // list positions [q0, q1): each list is sorted by key within the node, so
  // its first and last items hold the node's smallest and largest key
  auto tight_dim = [&](uint32_t sl, uint32_t q0, uint32_t q1) -> int {
    uint32_t lo[3], hi[3];
    for (int d = 0; d < k; ++d) {
      const uint16_t* list = s_lists + (size_t)slot_of(sl, d) * kLocalCap;
      const uint4 e0 = key_of[list[q0]], e1 = key_of[list[q1 - 1]];
      lo[d] = d == 0 ? e0.x : (d == 1 ? e0.y : e0.z);
      hi[d] = d == 0 ? e1.x : (d == 1 ? e1.y : e1.z);
    }
    return widest_of_keys(lo, hi, k, a.ctype);
  };
  // per depth jj below the block's root (level l0 + jj): the block's layout,
  // the round-robin split dimension and the lists read on deeper levels,
  // computed once
  __shared__ Local s_lay[kLocalLog + 1];
  __shared__ uint8_t s_drr[kLocalLog + 1], s_need[kLocalLog + 1];
  const int depths = tree.L - l0;  // levels l0 .. tree.L - 1
  if (depths > kLocalLog + 1) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_INTERNAL);
    return;
  }
  if (threadIdx.x < (unsigned)depths) {
    const int jj = threadIdx.x, L = l0 + jj;
    s_lay[jj] = make_local(tree, L, wk.s_rel << jj, 1u << jj);
    const int dr = L % k;
    s_drr[jj] = (uint8_t)dr;
    uint32_t need = bydim ? (1u << k) - 1u : 0u;
    int md = dr + 1 == k ? 0 : dr + 1;
    for (int q = L + 1, c = 0; q <= tree.L - 1 && c < k; ++q, ++c) {
      need |= 1u << md;
      md = md + 1 == k ? 0 : md + 1;
    }
    s_need[jj] = (uint8_t)need;
  }
  __syncthreads();
  // Tag update of depth jj (Sec. 3.2 with Observation 1) for the segments
  // [r.uf, r.uf + cnt) of range r: in its segment the item at rank pr (the
  // left subtree's size) is pinned as the node, lower ranks go left, higher
  // ranks right.  Each item gets an info word (side << 14 | offset); the
  // offset is its position on the next level minus its rank among the
  // range's items of the same side in list order: left items of a segment go
  // after the right items of the range's earlier segments, right items after
  // the left items of the earlier segments and of the segment itself.  The
  // pivots are pinned and (clipped-domain rule) their planes recorded.  The
  // range's items are stored from list position sb on.
  //
  // The `gs` threads of a group (g0 = index in the group) take whole
  // segments: with at least as many threads as segments, 2^x threads share
  // one segment; with fewer, each thread takes every gs-th segment.  Either
  // way a segment's constants (start, pivot rank, next-level offsets of its
  // two sides, from the closed forms of Sec. 4) are computed once per thread
  // and segment, not once per item.
  auto info_pass = [&](const Range& r, uint32_t cnt, uint32_t jj, int L, uint32_t slots, uint32_t sb,
                       uint32_t g0, uint32_t gs) {
    const int drr = s_drr[jj];
    const uint32_t dbase = (1u << jj) - 1;  // local index of the first node at depth jj
    const Local& y = r.y;
    const uint32_t tps = gs >= cnt ? gs / cnt : 1u;  // threads per segment
    const uint32_t u0 = gs >= cnt ? g0 / tps : g0, ustep = gs >= cnt ? cnt : gs;
    const uint32_t t0 = gs >= cnt ? g0 % tps : 0u;
    for (uint32_t uu = u0; uu < cnt; uu += ustep) {
      const uint32_t tl = r.uf + uu;
      const uint32_t st = l_start(y, tl), en = l_start(y, tl + 1);
      uint32_t pr = 0, sl = 0;
      if (y.h >= 1) {
        pr = l_left(y, tl);
        sl = l_left_before(y, tl) - r.lb0;
      }
      const uint32_t sr = (st - r.p0) - uu - sl;
      const uint32_t offl = r.nb + sr, offr = r.nb + sl + pr;
      const int d = bydim ? s_ldim[dbase + tl] : drr;
      const uint16_t* list = s_lists + (size_t)slot_of(slots, d) * kLocalCap;
      for (uint32_t p = st + t0; p < en; p += tps) {
        const uint32_t q = p - st;
        const uint32_t side = q < pr ? 0u : (q == pr ? 2u : 1u);
        const uint32_t off = side == 0 ? offl : (side == 1 ? offr : 0u);
        const uint32_t it = list[p - r.p0 + sb];
        if (it >= m || off >= kLocalCap) {
          s_bad = 1;
          continue;
        }
        s_info[it] = (uint16_t)((side << 14) | off);
      }
      // the group's first thread pins the segment's pivot: with one thread
      // per segment, the lanes of a warp write consecutive nodes together
      if (t0 == 0 && st + pr < en) {
        const uint32_t it = list[st + pr - r.p0 + sb];
        if (it >= m) {
          s_bad = 1;
          continue;
        }
        const uint32_t o = s_orig[it];
        const uint32_t node = ls.off + full_nodes(L) + (wk.s_rel << jj) + tl;
        a.perm[node] = o;
        if (ent_of) {  // the record goes straight to its node
          const uint4 e = ent_of[it];
          write_record_from_entry(a.pts_out + (uint64_t)node * a.stride, e, k, a.ctype);
          if (widest)
            s_lplane[dbase + tl] =
                __uint_as_float(key_to_float_bits(d == 0 ? e.x : (d == 1 ? e.y : e.z)));
        } else if (widest) {
          s_lplane[dbase + tl] = coord_of(a.pts, o, a.stride, d);
        }
      }
    }
  };

  uint32_t slots = 0;
  for (int q = 0; q <= k; ++q) slots |= (uint32_t)q << (4 * q);
  constexpr int PER = kLocalCap / T;  // positions per thread in a block-wide partition

  for (uint32_t j = 0;; ++j) {
    const int L = l0 + (int)j;
    if (L > tree.L - 1) break;
    const uint32_t nodes = 1u << j;
    const uint32_t first = wk.s_rel << j;
    const Local& yj = s_lay[j];
    if (nodes >= (uint32_t)W) {
      // From here every subtree of depth j is finished by one warp.  On every
      // later level the warp keeps its subtree's items from the subtree's
      // start at depth j on (the set of items only shrinks), so no other
      // warp touches them and warps need no block barrier.
      for (uint32_t tw = warp; tw < nodes; tw += W) {
        uint32_t wslots = slots;
        const uint32_t sb = l_start(yj, tw);
        for (uint32_t i = 0;; ++i) {
          const int Li = L + (int)i;
          if (Li > tree.L - 1) break;
          const uint32_t jj = j + i;
          const uint32_t firsti = wk.s_rel << jj;
          const uint32_t cnt = 1u << i;
          const Range r = make_range(s_lay[jj], tw << i, cnt);
          if (r.p0 >= r.p1) break;
          if (bydim) {
            for (uint32_t u = lane; u < cnt; u += 32) {
              const uint32_t tl = (tw << i) + u;
              const uint32_t node = full_nodes(Li) + firsti + tl;
              if (node >= tree.n) continue;
              const int d = widest ? node_dim(jj, tl)
                                   : tight_dim(wslots, l_start(s_lay[jj], tl) - r.p0 + sb,
                                               l_start(s_lay[jj], tl + 1) - r.p0 + sb);
              s_ldim[(1u << jj) - 1 + tl] = (uint8_t)d;
              a.dims[ls.off + node] = (uint8_t)d;
            }
            __syncwarp();
          }
          info_pass(r, cnt, jj, Li, wslots, sb, lane, 32);
          __syncwarp();
          if (Li == tree.L - 1) break;
          const uint32_t lim = r.nb + (r.p1 - r.p0) - cnt;  // end of the range's next-level items
          for (int d = 0; d < k; ++d) {
            if (!((s_need[jj] >> d) & 1u)) continue;
            const uint16_t* src = s_lists + (size_t)slot_of(wslots, d) * kLocalCap;
            uint16_t* dst = s_lists + (size_t)slot_of(wslots, k) * kLocalCap;
            uint32_t cl = 0, cr = 0;
            for (uint32_t b = r.p0; b < r.p1; b += 32) {
              const uint32_t p = b + lane;
              uint32_t it = 0, v = 3u << 14;
              if (p < r.p1) {
                it = src[p - r.p0 + sb];
                v = s_info[it];
              }
              const uint32_t side = v >> 14;
              const uint32_t bl = __ballot_sync(0xffffffffu, side == 0);
              const uint32_t br = __ballot_sync(0xffffffffu, side == 1);
              if (side < 2) {
                const uint32_t np =
                    (v & 0x3FFFu) + (side == 0 ? cl + __popc(bl & lt) : cr + __popc(br & lt));
                if (np >= r.nb && np < lim) dst[np - r.nb + sb] = (uint16_t)it;
                else s_bad = 1;
              }
              cl += __popc(bl);
              cr += __popc(br);
            }
            __syncwarp();
            wslots = swap_slots(wslots, d, k);
          }
        }
      }
      break;
    }
    const Range r = make_range(yj, 0, nodes);
    const uint32_t mj = r.p1;
    if ((widest && j > 0) || tight) {
      for (uint32_t tl = threadIdx.x; tl < nodes; tl += T) {
        const uint32_t node = full_nodes(L) + first + tl;
        if (node >= tree.n) continue;
        const int d = widest ? node_dim(j, tl) : tight_dim(slots, l_start(yj, tl), l_start(yj, tl + 1));
        s_ldim[(1u << j) - 1 + tl] = (uint8_t)d;
        a.dims[ls.off + node] = (uint8_t)d;
      }
      __syncthreads();
    }
    info_pass(r, nodes, j, L, slots, 0, threadIdx.x, T);
    __syncthreads();
    if (L == tree.L - 1) break;  // lowest level: every item was pinned
    const uint32_t mn = mj - nodes;
    // stable partition of every list still needed into the next level's
    // order: each warp ranks a contiguous chunk with ballots, one block
    // exchange of the warps' counts, then every item is written
    const uint32_t chunk = ((mj + W * 32 - 1) / (W * 32)) * 32;
    for (int d = 0; d < k; ++d) {
      if (!((s_need[j] >> d) & 1u)) continue;
      const uint16_t* src = s_lists + (size_t)slot_of(slots, d) * kLocalCap;
      uint16_t* dst = s_lists + (size_t)slot_of(slots, k) * kLocalCap;
      uint32_t its[PER], vs[PER];
      uint32_t cl = 0, cr = 0;
      const uint32_t c0 = (uint32_t)warp * chunk;
      const int rounds = (int)(chunk / 32);  // block-uniform
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        if (q >= rounds) break;
        const uint32_t p = c0 + (uint32_t)q * 32 + lane;
        uint32_t it = 0, v = 3u << 14;
        if (p < mj) {
          it = src[p];
          v = s_info[it];
        }
        const uint32_t side = v >> 14;
        const uint32_t bl = __ballot_sync(0xffffffffu, side == 0);
        const uint32_t br = __ballot_sync(0xffffffffu, side == 1);
        const uint32_t rank = side == 0 ? cl + __popc(bl & lt) : cr + __popc(br & lt);
        its[q] = it | (rank << 16);
        vs[q] = v;
        cl += __popc(bl);
        cr += __popc(br);
      }
      if (lane == 0) s_w[warp] = cl | (cr << 16);
      __syncthreads();
      const uint32_t before = __reduce_add_sync(0xffffffffu, lane < warp ? s_w[lane] : 0u);
      const uint32_t wl = before & 0xFFFFu, wr = before >> 16;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        if (q >= rounds) break;
        const uint32_t side = vs[q] >> 14;
        if (side > 1) continue;
        const uint32_t np = (vs[q] & 0x3FFFu) + (side == 0 ? wl : wr) + (its[q] >> 16);
        if (np < mn) dst[np] = (uint16_t)(its[q] & 0xFFFFu);
        else s_bad = 1;
      }
      __syncthreads();
      slots = swap_slots(slots, d, k);
    }
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
  const void* fn = a.mode == 1   ? (const void*)local_finish_kernel<1>
                   : a.mode == 2 ? (const void*)local_finish_kernel<2>
                                 : (const void*)local_finish_kernel<0>;
  cudaError_t e = ensure_smem(fn, smem);
  if (e != cudaSuccess) return e;
  if (a.mode == 1) local_finish_kernel<1><<<a.nwork, T, smem, st>>>(a);
  else if (a.mode == 2) local_finish_kernel<2><<<a.nwork, T, smem, st>>>(a);
  else local_finish_kernel<0><<<a.nwork, T, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace kdb
