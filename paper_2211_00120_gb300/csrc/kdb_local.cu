// kdb_local.cu -- finish small subtrees on chip.
//
// Once every subtree of a level holds at most 2^13 - 1 points, one thread
// block takes one subtree and runs all of its remaining levels in shared
// memory, writing only the final node -> point entries.
//
// Inside the block, each level still performs the paper's step: order every
// node's points by (tag, coordinate) (Sec. 3.1) and apply the tag update
// (Sec. 3.2).  The block keeps k lists of local ids, one per dimension, each
// sorted by (key_d, original index), and one tag per point: its node on the
// current level.  The points of a node are a subset of every list, in the
// list's order, so a point's rank among its node's points in the order of
// dimension d is the number of earlier entries of list d with the same tag.
// A level with split dimension d is therefore one pass over list d: each
// point gets that rank by counting (warp match_any, per-node counters), the
// point at rank ss(lChild) is pinned as the node (Observation 1), lower ranks
// go to the left child and higher ranks to the right one -- only the tags
// change, the lists are not re-sorted.
//
// The first levels run block-wide (per-warp counts, then an exclusive prefix
// over the warps for each node).  At the depth with 32 nodes every list is
// split once, stably, into the 32 nodes' runs; from then on each warp owns
// one node's points and finishes its subtree alone, with counters of its
// own and no block barrier.  The pinned points are recorded per node and
// written at the end, node by node, so that consecutive threads write
// consecutive nodes.
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
// or hash table (2 slots per item of 4 + 2 bytes); on the levels, per item a
// tag (2), per block node the pinned item, split dimension and plane (or
// tight-box corners) (2 + 1 + 4), and the counters (3)
static_assert(2 * kLocalCap * 4 + 2 * kLocalCap * 2 <= 12 * kLocalCap, "hash table fits");
constexpr int kJW = 5;                       // first depth of the warp phase: 2^5 = W nodes
constexpr int kWT = kLocalCap >> (kJW + 1);  // most nodes of one warp on a depth that splits
constexpr uint32_t kPin = 0xFFFFu;           // tag of a pinned item
constexpr uint32_t kMoved = 0x8000u;         // tag flag: already split on this depth
static_assert((1 << kJW) == W, "one warp per node of the first warp depth");
static_assert(2 * W * 32 * 4 <= 3 * kLocalCap && W * kWT * 4 <= 3 * kLocalCap, "counters fit");
static_assert(kLocalCap <= (1 << 13) && kLocalMax < (1 << 13), "ids and in-warp ranks pack in 13 bits");

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
      const uint32_t peers = warp_peers(d, ok, 8);
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

__device__ inline uint32_t comp3(const uint4& e, int d) {
  return d == 0 ? e.x : (d == 1 ? e.y : e.z);
}

// Tight-box rule, one dimension at a time: extent hi - lo of dimension d
// (float32, round to nearest; integers: the exact difference of the keys,
// which are ordered like the values) against the widest so far, scanned from
// d = 0 with a strict '>' (the lowest dimension wins ties), as for a whole box.
__device__ inline void tight_step(uint32_t lo, uint32_t hi, int d, int ctype, uint32_t* best,
                                  uint8_t* dim) {
  if (ctype != kCoordF32) {
    const uint32_t e = hi - lo;
    if (d == 0 || e > *best) {
      *best = e;
      *dim = (uint8_t)d;
    }
    return;
  }
  const float e = __fsub_rn(__uint_as_float(key_to_float_bits(hi)), __uint_as_float(key_to_float_bits(lo)));
  if (d == 0 || e > __uint_as_float(*best)) {
    *best = __float_as_uint(e);
    *dim = (uint8_t)d;
  }
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
  uint16_t* s_tag = reinterpret_cast<uint16_t*>(s_area);                   // per item: its node
  uint16_t* s_pin = s_tag + kLocalCap;                                      // per block node: its item
  uint8_t* s_ldim = reinterpret_cast<uint8_t*>(s_pin + kLocalCap);         // per block node
  float* s_lplane = reinterpret_cast<float*>(s_ldim + kLocalCap);          // per block node
  uint32_t* s_ctr = reinterpret_cast<uint32_t*>(s_lplane + kLocalCap);     // counters
  // tight-box rule, in place of the planes: per node of the current depth
  // the items holding its smallest and largest key of one dimension, and its
  // widest extent so far (a splitting depth has at most cap / 2 nodes)
  uint16_t* s_tlo = reinterpret_cast<uint16_t*>(s_lplane);
  uint16_t* s_thi = s_tlo + kLocalCap / 2;
  uint32_t* s_tbest = reinterpret_cast<uint32_t*>(s_thi + kLocalCap / 2);

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
  if (l0 > 0) dpar = kMode == 0 ? (l0 - 1 + a.dim0) % k : a.dims[ls.off + (s0 - 1) / 2];
  uint16_t* s_wh = s_lists + (size_t)k * kLocalCap;  // radix counters (spare list slot)
  if (a.lorig && l0 > 0) {
    // The global passes hand over every list of the subtree as original
    // indices, already in order.  Local id = position in list 0; the other
    // lists are translated through a hash table original index -> local id.
    const uint32_t* lo0 = a.lorig + ls.off + start0;
    const uint4* le0 = a.lents ? a.lents + ls.off + start0 : nullptr;  // list 0 as entries
    constexpr uint32_t HM = 2 * kLocalCap - 1;
    constexpr int PER = kLocalCap / T;  // items per thread (8)
    if (k > 3) s_bad = 1;  // lists are handed over for k <= 3 only
    // every thread's items of every list are loaded at once, so that their
    // global loads are in flight together
    uint32_t ov[3][PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const uint32_t i = threadIdx.x + (uint32_t)r * T;
      ov[0][r] = ov[1][r] = ov[2][r] = 0;
      if (i < m) {
        ov[0][r] = le0 ? reinterpret_cast<const uint32_t*>(le0 + i)[3] : lo0[i];
        if (k > 1) ov[1][r] = a.lorig[(size_t)a.total + ls.off + start0 + i];
        if (k > 2) ov[2][r] = a.lorig[(size_t)2 * a.total + ls.off + start0 + i];
      }
    }
    for (uint32_t i = threadIdx.x; i < 2 * kLocalCap; i += T) s_hkey[i] = 0xFFFFFFFFu;
    __syncthreads();
    // Inserts in rounds, without atomics: every pending item writes its key
    // into the first empty slot it sees from its probe position on; after a
    // barrier the item whose key is in the slot owns it, the others move on
    // to the next slot.  A slot owned in an earlier round is never empty
    // again, so no owner is displaced.
    uint32_t hh[PER];
    uint32_t pend = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const uint32_t i = threadIdx.x + (uint32_t)r * T;
      hh[r] = 0;
      if (i >= m) continue;
      if (ov[0][r] >= a.total) {
        s_bad = 1;
        ov[0][r] = 0;
      }
      s_orig[i] = ov[0][r];
      s_lists[i] = (uint16_t)i;
      hh[r] = (ov[0][r] * 0x9E3779B1u) >> (32 - (kLocalLog + 1));
      pend |= 1u << r;
    }
    for (int round = 0; round < 64; ++round) {
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        if (!((pend >> r) & 1u)) continue;
        uint32_t h = hh[r];
        for (uint32_t probe = 0; probe <= HM; ++probe) {
          const uint32_t key = s_hkey[h];
          if (key == 0xFFFFFFFFu) break;
          if (key == ov[0][r]) s_bad = 1;  // the key is owned already: an original index twice
          h = (h + 1) & HM;
        }
        hh[r] = h;
        s_hkey[h] = ov[0][r];
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        if (!((pend >> r) & 1u)) continue;
        if (s_hkey[hh[r]] == ov[0][r]) {
          s_hval[hh[r]] = (uint16_t)(threadIdx.x + (uint32_t)r * T);
          pend &= ~(1u << r);
        } else {
          hh[r] = (hh[r] + 1) & HM;
        }
      }
      if (!__syncthreads_or(pend != 0u)) break;
    }
    if (pend) s_bad = 1;
    __syncthreads();
    // an original index twice (corrupt input lists): two items own one slot
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const uint32_t i = threadIdx.x + (uint32_t)r * T;
      if (i < m && s_hval[hh[r]] != (uint16_t)i) s_bad = 1;
    }
#pragma unroll
    for (int d = 1; d < 3; ++d) {
      if (d >= k) break;
      uint16_t* list = s_lists + (size_t)d * kLocalCap;
      // lookups: every item's first probe is read at once (most keys sit in
      // their first slot), then each probe runs on to the key or an empty
      // slot, then the ids are read
      uint32_t key[PER];
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        hh[r] = (ov[d][r] * 0x9E3779B1u) >> (32 - (kLocalLog + 1));
        key[r] = s_hkey[hh[r]];
      }
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const uint32_t i = threadIdx.x + (uint32_t)r * T;
        if (i >= m) continue;
        const uint32_t o = ov[d][r];
        uint32_t h = hh[r], kk = key[r];
        for (uint32_t probe = 0; probe < HM && kk != o && kk != 0xFFFFFFFFu; ++probe) {
          h = (h + 1) & HM;
          kk = s_hkey[h];
        }
        hh[r] = kk == o ? h : 0xFFFFFFFFu;
      }
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const uint32_t i = threadIdx.x + (uint32_t)r * T;
        if (i >= m) continue;
        uint32_t id = hh[r] != 0xFFFFFFFFu ? (uint32_t)s_hval[hh[r]] : 0xFFFFFFFFu;
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
      s_ldim[0] = (uint8_t)widest_dim(s_box, s_box + kMaxK, k);
    } else {
      const float* b = a.boxes_local + ((size_t)ls.lbox0 + wk.s_rel) * 2 * k;
      for (int d = 0; d < k; ++d) {
        s_box[d] = b[d];
        s_box[kMaxK + d] = b[k + d];
      }
      s_ldim[0] = a.dims[ls.off + s0];
    }
  }

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
  // split dimension of block node tl at depth jj: widest side of its domain,
  // the root's domain clipped by the planes of its ancestors inside the block
  // (Sec. 6)
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
  // per depth jj below the block's root (level l0 + jj): the block's layout
  // and the round-robin split dimension, computed once
  __shared__ Local s_lay[kLocalLog + 1];
  __shared__ uint8_t s_drr[kLocalLog + 1];
  __shared__ uint32_t s_prb[W];  // block phase: pivot rank (and size) of each node
  __shared__ uint32_t s_szb[W];
  const int depths = tree.L - l0;  // levels l0 .. tree.L - 1
  if (depths > kLocalLog + 1 || depths < 1) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_INTERNAL);
    return;
  }
  if (threadIdx.x < (unsigned)depths) {
    const int jj = threadIdx.x, L = l0 + jj;
    s_lay[jj] = make_local(tree, L, wk.s_rel << jj, 1u << jj);
    s_drr[jj] = (uint8_t)((L + a.dim0) % k);
  }
  for (uint32_t i = threadIdx.x; i < kLocalCap; i += T) {
    if (i < m) s_tag[i] = 0;  // every item starts in the root
    s_pin[i] = (uint16_t)kPin;
  }
  s_ctr[threadIdx.x] = 0;  // block counters [W][32]
  __syncthreads();

  // The pivot of node t at depth jj: its item is recorded, its plane kept for
  // the children's domains (clipped-domain rule).
  auto pin = [&](uint32_t id, uint32_t jj, uint32_t t, int d) {
    const uint32_t hn = (1u << jj) - 1 + t;
    s_pin[hn] = (uint16_t)id;
    if (widest)
      s_lplane[hn] = ent_of ? __uint_as_float(key_to_float_bits(comp3(ent_of[id], d)))
                            : coord_of(a.pts, s_orig[id], a.stride, d);
  };
  uint32_t slots = 0;
  for (int q = 0; q <= k; ++q) slots |= (uint32_t)q << (4 * q);
  auto list_of = [&](uint32_t sl, int d) -> uint16_t* {
    return s_lists + (size_t)slot_of(sl, d) * kLocalCap;
  };

  // Block-wide pass over list `list` at depth j (at most W nodes): every item
  // whose node splits in dimension d (every live item if d < 0) gets its
  // rank among its node's items in the list's order -- per-warp counts of
  // each node over contiguous chunks of the list, then for each node an
  // exclusive prefix over the warps -- and use(id, t, rank) is called.
  constexpr int PER = kLocalCap / T;  // positions per thread (8)
  auto block_ranks = [&](const uint16_t* list, uint32_t j, int d, auto&& use) {
    uint32_t* s_bc = s_ctr;           // [W][32] items per warp and node
    uint32_t* s_bb = s_ctr + W * 32;  // [W][32] items of the node in earlier warps
    const uint32_t nodes = 1u << j;
    const uint32_t nb = nodes - 1;
    const uint32_t chunk = ((m + W * 32 - 1) / (W * 32)) * 32;
    const int rounds = (int)(chunk / 32);  // block-uniform
    const uint32_t c0 = (uint32_t)warp * chunk;
    uint32_t pk[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      pk[q] = 0xFFFFFFFFu;
      if (q >= rounds) continue;
      const uint32_t p = c0 + (uint32_t)q * 32 + lane;
      uint32_t t = kPin, id = 0;
      if (p < m) {
        id = list[p];
        t = s_tag[id];
        if (t >= kMoved || (d >= 0 && s_ldim[nb + t] != d)) t = kPin;
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, t);
      uint32_t before = 0;
      if (t != kPin) before = s_bc[warp * 32 + t];
      __syncwarp();
      if (t != kPin) {
        if ((peers & lt) == 0) s_bc[warp * 32 + t] = before + __popc(peers);
        pk[q] = ((before + __popc(peers & lt)) << 18) | (t << 13) | id;
      }
      __syncwarp();
    }
    __syncthreads();
    if ((uint32_t)warp < nodes) {  // warp t: node t's counts over the warps
      const uint32_t v = s_bc[lane * 32 + warp];
      uint32_t x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      s_bb[lane * 32 + warp] = x - v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      if (pk[q] == 0xFFFFFFFFu) continue;
      const uint32_t id = pk[q] & 0x1FFFu, t = (pk[q] >> 13) & 31u;
      use(id, t, s_bb[warp * 32 + t] + (pk[q] >> 18));
    }
    s_bc[threadIdx.x] = 0;  // for the next pass
    __syncthreads();
  };
  // tag update of one item at depth jj from its rank r in its node t
  // (Sec. 3.2 with Observation 1): the children of block node t are 2t, 2t+1.
  // With a split dimension per node, a depth takes one pass per dimension:
  // the new tag is flagged so that the later passes of the depth skip it.
  constexpr uint32_t kFlag = bydim ? kMoved : 0u;
  auto split_item = [&](uint32_t id, uint32_t jj, uint32_t t, uint32_t r, uint32_t pr, int d) {
    if (r < pr) s_tag[id] = (uint16_t)((2 * t) | kFlag);
    else if (r > pr) s_tag[id] = (uint16_t)((2 * t + 1) | kFlag);
    else {
      s_tag[id] = (uint16_t)kPin;
      pin(id, jj, t, d);
    }
  };

  const int D = depths;
  const int jb = D - 1 < kJW ? D - 1 : kJW;  // block phase: depths 0 .. jb-1 (the last one is leaves)
  int jfirst = 0;
  if (jb > 0) {
    // depth 0: one node holds every item, so an item's rank in it is its
    // position in the list
    if (tight) {
      if (threadIdx.x == 0)
        for (int d = 0; d < k; ++d) {
          const uint16_t* ld = list_of(slots, d);
          tight_step(comp3(key_of[ld[0]], d), comp3(key_of[ld[m - 1]], d), d, a.ctype, &s_tbest[0],
                     &s_ldim[0]);
        }
      __syncthreads();
    }
    const int d0 = bydim ? (int)s_ldim[0] : (int)s_drr[0];
    const uint32_t pr0 = l_left(s_lay[0], 0);
    const uint16_t* ld = list_of(slots, d0);
    for (uint32_t p = threadIdx.x; p < m; p += T) {
      const uint32_t id = ld[p];
      if (p < pr0) s_tag[id] = 0;
      else if (p > pr0) s_tag[id] = 1;
      else {
        s_tag[id] = (uint16_t)kPin;
        pin(id, 0, 0, d0);
      }
    }
    __syncthreads();
    jfirst = 1;
  }
  // lists already split into the runs of depth kJW's nodes (see below)
  uint32_t split5 = 0;
  for (int j = jfirst; j < jb; ++j) {
    const Local& y = s_lay[j];
    const uint32_t nodes = 1u << j, nb = nodes - 1;
    if (threadIdx.x < nodes) {
      s_prb[threadIdx.x] = l_left(y, threadIdx.x);
      s_szb[threadIdx.x] = l_start(y, threadIdx.x + 1) - l_start(y, threadIdx.x);
      if (widest && j > 0) s_ldim[nb + threadIdx.x] = (uint8_t)node_dim(j, threadIdx.x);
    }
    __syncthreads();
    if (tight) {
      // the box of every node: in list d its first and last items hold its
      // smallest and largest key_d
      for (int d = 0; d < k; ++d) {
        block_ranks(list_of(slots, d), j, -1, [&](uint32_t id, uint32_t t, uint32_t r) {
          if (r == 0) s_tlo[t] = (uint16_t)id;
          if (r + 1 == s_szb[t]) s_thi[t] = (uint16_t)id;
        });
        if (threadIdx.x < nodes)
          tight_step(comp3(key_of[s_tlo[threadIdx.x]], d), comp3(key_of[s_thi[threadIdx.x]], d), d,
                     a.ctype, &s_tbest[threadIdx.x], &s_ldim[nb + threadIdx.x]);
        __syncthreads();
      }
    }
    // round robin, the last block depth before the warp phase: an item's
    // rank in its child follows from its rank in its node (Observation 1:
    // lower ranks go left in order, higher ones right), so this pass also
    // writes the list in the runs of depth kJW's nodes, and the split before
    // the warp phase skips it
    const bool split_here = !bydim && j == kJW - 1 && D - 1 > kJW;
    for (int d = 0; d < k; ++d) {
      if (!bydim && d != s_drr[j]) continue;
      if (split_here) {
        uint16_t* dst = list_of(slots, k);
        const Local& y5 = s_lay[kJW];
        block_ranks(list_of(slots, d), j, -1, [&](uint32_t id, uint32_t t, uint32_t r) {
          const uint32_t pr = s_prb[t];
          split_item(id, j, t, r, pr, d);
          if (r != pr) {
            const uint32_t pos = r < pr ? l_start(y5, 2 * t) + r : l_start(y5, 2 * t + 1) + (r - pr - 1);
            if (pos < kLocalCap) dst[pos] = (uint16_t)id;
            else s_bad = 1;
          }
        });
        slots = swap_slots(slots, d, k);
        split5 |= 1u << d;
        continue;
      }
      block_ranks(list_of(slots, d), j, bydim ? d : -1, [&](uint32_t id, uint32_t t, uint32_t r) {
        split_item(id, j, t, r, s_prb[t], d);
      });
    }
    if (bydim) {  // clear the flags of the depth
      for (uint32_t id = threadIdx.x; id < m; id += T) {
        const uint32_t t = s_tag[id];
        if (t != kPin) s_tag[id] = (uint16_t)(t & ~kMoved);
      }
      __syncthreads();
    }
  }

  if (D - 1 > kJW) {
    // every list read on a warp depth is split into the runs of the 32 nodes
    // of depth kJW, in the layout of that depth (pinned items dropped)
    uint32_t need = bydim ? (1u << k) - 1u : 0u;
    if (!bydim)
      for (int jj = kJW; jj < D - 1; ++jj) need |= 1u << s_drr[jj];
    const Local& y5 = s_lay[kJW];
    for (int d = 0; d < k; ++d) {
      if (!((need >> d) & 1u) || ((split5 >> d) & 1u)) continue;
      uint16_t* dst = list_of(slots, k);
      block_ranks(list_of(slots, d), kJW, -1, [&](uint32_t id, uint32_t t, uint32_t r) {
        const uint32_t pos = l_start(y5, t) + r;
        if (pos < kLocalCap) dst[pos] = (uint16_t)id;
        else s_bad = 1;
      });
      slots = swap_slots(slots, d, k);
    }
    // warp phase: warp w finishes node w of depth kJW
    const uint32_t wb = l_start(y5, warp), we = l_start(y5, warp + 1);
    // per node of the warp: pivot rank << 16 | items counted so far
    uint32_t* wc = s_ctr + warp * kWT;
    // One warp's pass over its run of list `list` at depth jj: every item
    // whose node splits in dimension d (all if d < 0) gets its rank among its
    // node's items in list order (the warp holds all of them, so a running
    // count per node is the rank).
    // (each item is in the run once, so reading the next round's item and
    // tag ahead of this round's tag updates reads nothing they write)
    auto warp_ranks = [&](const uint16_t* list, uint32_t jj, uint32_t tb, int d, auto&& use) {
      const uint32_t nb = (1u << jj) - 1, nloc = 1u << (jj - kJW);
      uint32_t nid = 0, ntag = kPin;
      if (wb + lane < we) {
        nid = list[wb + lane];
        ntag = s_tag[nid];
      }
      for (uint32_t b = wb; b < we; b += 32) {
        const uint32_t id = nid, t = ntag;
        ntag = kPin;
        if (b + 32 + lane < we) {
          nid = list[b + 32 + lane];
          ntag = s_tag[nid];
        }
        uint32_t u = kPin;
        if (t < kMoved && (d < 0 || s_ldim[nb + t] == d)) u = t - tb;
        if (u != kPin && u >= nloc) {  // not this warp's: inconsistent lists
          s_bad = 1;
          u = kPin;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, u);
        uint32_t w = 0;
        if (u != kPin) w = wc[u];
        __syncwarp();
        if (u != kPin) {
          if ((peers & lt) == 0) wc[u] = w + __popc(peers);
          use(id, u, (w & 0xFFFFu) + __popc(peers & lt), w >> 16);
        }
        __syncwarp();
      }
    };
    for (int jj = kJW; jj < D - 1; ++jj) {
      const Local& y = s_lay[jj];
      const uint32_t i = (uint32_t)(jj - kJW), nloc = 1u << i, tb = (uint32_t)warp << i;
      const uint32_t nb = (1u << jj) - 1;
      if (nloc > (uint32_t)kWT) {
        s_bad = 1;
        break;
      }
      for (uint32_t u = lane; u < nloc; u += 32) {
        wc[u] = l_left(y, tb + u) << 16;
        if (widest) s_ldim[nb + tb + u] = (uint8_t)node_dim(jj, tb + u);
      }
      __syncwarp();
      if (tight) {
        for (int d = 0; d < k; ++d) {
          warp_ranks(list_of(slots, d), jj, tb, -1, [&](uint32_t id, uint32_t u, uint32_t r, uint32_t) {
            const uint32_t t = tb + u;
            if (r == 0) s_tlo[t] = (uint16_t)id;
            if (r + 1 == l_start(y, t + 1) - l_start(y, t)) s_thi[t] = (uint16_t)id;
          });
          for (uint32_t u = lane; u < nloc; u += 32) {
            const uint32_t t = tb + u;
            tight_step(comp3(key_of[s_tlo[t]], d), comp3(key_of[s_thi[t]], d), d, a.ctype, &s_tbest[t],
                       &s_ldim[nb + t]);
            wc[u] &= 0xFFFF0000u;
          }
          __syncwarp();
        }
      }
      for (int d = 0; d < k; ++d) {
        if (!bydim && d != s_drr[jj]) continue;
        warp_ranks(list_of(slots, d), jj, tb, bydim ? d : -1,
                   [&](uint32_t id, uint32_t u, uint32_t r, uint32_t pr) { split_item(id, jj, tb + u, r, pr, d); });
      }
      if (bydim) {  // clear the flags of the warp's items
        const uint16_t* l0s = list_of(slots, 0);
        for (uint32_t p = wb + lane; p < we; p += 32) {
          const uint32_t id = l0s[p], t = s_tag[id];
          if (t != kPin) s_tag[id] = (uint16_t)(t & ~kMoved);
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // the lowest depth: every item left is a leaf, its node is its tag
  {
    const uint32_t nb = (1u << (D - 1)) - 1, nodes = 1u << (D - 1);
    for (uint32_t id = threadIdx.x; id < m; id += T) {
      const uint32_t t = s_tag[id];
      if (t == kPin) continue;
      if (t < nodes) s_pin[nb + t] = (uint16_t)id;
      else s_bad = 1;
    }
  }
  __syncthreads();
  // every node of the block's subtree, in heap order (block node q is depth
  // jj = level(q), index q + 1 - 2^jj there): consecutive threads write
  // consecutive nodes (perm, the record, the split dimension); each thread
  // reads what four nodes need before it writes, so that the reads are in
  // flight together
  {
    const uint32_t hnodes = (1u << D) - 1;
    for (uint32_t q0 = threadIdx.x; q0 < hnodes; q0 += 4 * T) {
      uint32_t node[4], o[4], dd[4];
      uint4 e[4];
      bool ok[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t q = q0 + (uint32_t)r * T;
        ok[r] = false;
        if (q >= hnodes) continue;
        const int jj = level_of(q);
        const uint32_t t = q + 1 - (1u << jj);
        const uint32_t first = full_nodes(l0 + jj) + (wk.s_rel << jj);  // the depth's first node
        if (first + t >= tree.n) continue;
        const uint32_t id = s_pin[q];
        if (id >= m) {
          s_bad = 1;
          continue;
        }
        ok[r] = true;
        node[r] = ls.off + first + t;
        o[r] = s_orig[id];
        if (ent_of) e[r] = ent_of[id];
        if (bydim) {
          if (jj + 1 < D) dd[r] = s_ldim[q];
          else if (widest) dd[r] = jj == 0 ? s_ldim[0] : (uint32_t)node_dim(jj, t);
          else dd[r] = 0;  // tight box of a leaf: one point, every extent 0
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (!ok[r]) continue;
        a.perm[node[r]] = o[r];
        if (ent_of) write_record_from_entry(a.pts_out + (uint64_t)node[r] * a.stride, e[r], k, a.ctype);
        if (bydim) a.dims[node[r]] = (uint8_t)dd[r];
      }
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
