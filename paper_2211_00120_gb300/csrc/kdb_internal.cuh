// kdb_internal.cuh -- shared device/host helpers of the k-d tree builder.
//
// Implicit-tree arithmetic of the paper (Wald, arXiv 2211.00120):
//   level(i) = 31 - clz(i+1), L = numLevels(N) = 32 - clz(N), F(l) = 2^l - 1
//   (Sec. 2, with the Revision 3 correction of L); subtree size ss(s) in O(1)
//   (Sec. 4.1); segment begin sb(s,l) in O(1) (Sec. 4.2).  All arithmetic is
//   unsigned (the paper's ~((~s) << h) is undefined on signed ints).
//
// "Compacted" level arrays: after the level-l tag update every node of levels
// < l+1 is final, so the live points of level l+1 are kept in an array of
// N - F(l+1) items with the pinned nodes removed.  Segment (subtree) s_rel =
// s - F(l) of level l starts at sb(s,l) - F(l) in the level-l array.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kdb {

enum : uint32_t { ERR_NAN = 1u, ERR_TIMEOUT = 2u, ERR_INTERNAL = 4u };

constexpr int kMaxK = 8;
constexpr int kRadixBins = 256;  // 8-bit radix digits
constexpr uint32_t kMark = 0x80000000u;  // visited flag in the permutation array

__host__ __device__ inline int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz(x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

__host__ __device__ inline int num_levels(uint32_t n) { return 32 - clz32(n); }
__host__ __device__ inline int level_of(uint32_t i) { return 31 - clz32(i + 1); }
__host__ __device__ inline uint32_t full_nodes(int l) { return (uint32_t)((1ull << l) - 1); }
// bits needed to hold values in [0, n)
__host__ __device__ inline int bits_for(uint64_t n) {
  int b = 0;
  while (b < 63 && (1ull << b) < n) ++b;
  return b;
}

struct Tree {
  uint32_t n;  // N
  int L;       // number of levels
  uint32_t m;  // nodes on the lowest level, N - F(L-1)
};

__host__ __device__ inline Tree make_tree(uint32_t n) {
  Tree t;
  t.n = n;
  t.L = n ? num_levels(n) : 0;
  t.m = n ? n - full_nodes(t.L - 1) : 0;
  return t;
}

// ss(s), Sec. 4.1: full inner levels below s plus its share of the lowest
// level.  0 for nodes outside the tree.
__host__ __device__ inline uint32_t subtree_size(const Tree& t, uint32_t s) {
  if (s >= t.n) return 0;
  const int h = t.L - level_of(s) - 1;
  const uint64_t w = 1ull << h;
  const uint64_t fllc = ((uint64_t)s << h) + (w - 1);  // first lowest-level child
  const uint64_t low = fllc >= t.n ? 0 : ((uint64_t)t.n - fllc < w ? (uint64_t)t.n - fllc : w);
  return (uint32_t)((w - 1) + low);
}

// Segment layout of level l (0 <= l <= L-2) in its compacted array.
// With h = L-l-1 >= 1 every subtree of level l has 2^h - 1 inner nodes and
// 0..2^h lowest-level nodes; the lowest level is filled from the left, so the
// first q subtrees are full (2^(h+1)-1), subtree q is partial and the rest
// are thin (2^h - 1) (Observation 3 together with Sec. 4.2).
struct LevelLayout {
  uint32_t m;      // lowest-level nodes of the whole tree
  int l, h;
  uint32_t full;   // 2^(h+1) - 1
  uint32_t thin;   // 2^h - 1
  uint32_t q;      // number of full subtrees
  uint32_t a;      // q * full: items covered by the full subtrees
  uint32_t part;   // size of subtree q (if q < 2^l)
  uint32_t nseg;   // 2^l
  uint32_t items;  // N - F(l)

  __host__ __device__ static LevelLayout make(const Tree& t, int l) {
    LevelLayout y;
    y.m = t.m;
    y.l = l;
    y.h = t.L - l - 1;
    y.thin = (uint32_t)((1ull << y.h) - 1);
    y.full = (uint32_t)((1ull << (y.h + 1)) - 1);
    y.nseg = 1u << l;
    uint32_t q = t.m >> y.h;
    y.q = q < y.nseg ? q : y.nseg;
    y.a = y.q * y.full;
    y.part = y.thin + (t.m - (y.q << y.h));  // only meaningful if q < nseg
    y.items = t.n - full_nodes(l);
    return y;
  }
  // sb(F(l) + s_rel, l) - F(l), Sec. 4.2
  __host__ __device__ uint32_t seg_start(uint32_t s_rel) const {
    const uint64_t lowest = (uint64_t)s_rel << h;
    return (uint32_t)((uint64_t)s_rel * thin + (lowest < m ? lowest : m));
  }
  // subtree of the item at compacted position j (inverse of seg_start)
  __host__ __device__ uint32_t seg_of(uint32_t j) const {
    if (j < a) return j / full;
    const uint32_t j2 = j - a;
    if (j2 < part) return q;
    return q + 1 + (j2 - part) / thin;
  }
  // ss(lChild(s)) for s = F(l) + s_rel: size of the left child's subtree,
  // which is the pivot rank of Observation 1
  __host__ __device__ uint32_t left_size(uint32_t s_rel) const {
    // left child is subtree 2*s_rel of level l+1 (h-1 levels below it)
    const int hc = h - 1;
    const uint64_t lowest = (uint64_t)(2 * s_rel) << hc;
    const uint64_t w = 1ull << hc;
    const uint64_t low = lowest >= m ? 0 : (m - lowest < w ? m - lowest : w);
    return (uint32_t)((w - 1) + low);
  }
  // sum of left_size(u) over u < x (h >= 1): every left child holds w - 1
  // upper nodes plus its share of the lowest level, which fills left to right
  __host__ __device__ uint32_t left_before(uint32_t x) const {
    const uint64_t w = 1ull << (h - 1);
    const uint64_t full = (uint64_t)m >> h;  // left children whose part of the lowest level is full
    uint64_t low = (x < full ? x : full) * w;
    if (x > full) {
      const uint64_t rest = (uint64_t)m - 2 * w * full;
      low += rest < w ? rest : w;
    }
    return (uint32_t)((uint64_t)x * (w - 1) + low);
  }
};

// Order-preserving map float32 -> uint32: unsigned order of the result is the
// float order with -0 < +0 (Sec. 7.1 suggests radix keys built from the
// coordinate bits; this is the usual sign-flip transform).
__host__ __device__ inline uint32_t float_key(uint32_t bits) {
  return bits ^ ((bits & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u);
}
__host__ __device__ inline uint32_t key_to_float_bits(uint32_t key) {
  return key ^ ((key & 0x80000000u) ? 0x80000000u : 0xFFFFFFFFu);
}
// Coordinate types (the mode argument's KDB_COORDS_* flag): float32, int32,
// uint32.  int32: two's complement order is the unsigned order of the bits
// with the sign bit flipped; uint32: the bits are the key.
// Both integer maps are one XOR with a per-type constant, so that each map is
// a single choice between the float map and that XOR (the record writes of
// the local finish go out over the host link for mapped host buffers, where
// they are measurably sensitive to how their stores are scheduled).
enum : int { kCoordF32 = 0, kCoordI32 = 1, kCoordU32 = 2 };
__host__ __device__ inline uint32_t int_key_xor(int ctype) { return ctype == kCoordI32 ? 0x80000000u : 0u; }
__host__ __device__ inline uint32_t coord_key(uint32_t bits, int ctype) {
  return ctype != kCoordF32 ? bits ^ int_key_xor(ctype) : float_key(bits);
}
__host__ __device__ inline uint32_t key_to_coord_bits(uint32_t key, int ctype) {
  return ctype != kCoordF32 ? key ^ int_key_xor(ctype) : key_to_float_bits(key);
}
#ifdef __CUDACC__
// The record of a point from its entry (k <= 3 coordinate keys, no payload):
// the key map is a bijection, so the bits are the input's.
__device__ inline void write_record_from_entry(unsigned char* rec, const uint4& e, int k, int ctype) {
  uint32_t* r = reinterpret_cast<uint32_t*>(rec);
  r[0] = key_to_coord_bits(e.x, ctype);
  if (k > 1) r[1] = key_to_coord_bits(e.y, ctype);
  if (k > 2) r[2] = key_to_coord_bits(e.z, ctype);
}
// Widest side of a box whose corners are coordinate keys: float32 extents
// hi - lo (round to nearest, no contraction) or, for integer coordinates,
// exact 64-bit differences (of the keys, which differ by what the values
// differ by: both integer key maps add a constant modulo 2^32 and keep the
// order); scanned from d = 0 with a strict '>', so the lowest
// dimension wins ties (an extent that is NaN, inf - inf, never wins).
__device__ inline int widest_of_keys(const uint32_t* lo, const uint32_t* hi, int k, int ctype) {
  int best = 0;
  if (ctype != kCoordF32) {
    int64_t be = 0;
    for (int d = 0; d < k; ++d) {
      const int64_t e = (int64_t)hi[d] - (int64_t)lo[d];
      if (d == 0 || e > be) {
        be = e;
        best = d;
      }
    }
    return best;
  }
  float be = 0.0f;
  for (int d = 0; d < k; ++d) {
    const float e = __fsub_rn(__uint_as_float(key_to_float_bits(hi[d])),
                              __uint_as_float(key_to_float_bits(lo[d])));
    if (d == 0 || e > be) {
      be = e;
      best = d;
    }
  }
  return best;
}
#endif

#ifdef __CUDACC__
// The lanes of the warp whose (valid, v) equals this lane's, v < 2^nbits:
// one ballot for validity and one per bit of v.  With many distinct values
// in a warp this costs less than __match_any_sync, measured on GB300.
// nbits must be warp-uniform.
__device__ inline uint32_t warp_peers(uint32_t v, bool valid, int nbits) {
  const uint32_t vb = __ballot_sync(0xffffffffu, valid);
  uint32_t m = valid ? vb : ~vb;
  for (int b = 0; b < nbits; ++b) {
    const bool bit = (v >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bal : ~bal;
  }
  return m;
}
__device__ inline uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ inline uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// ---- TMA bulk copies (cp.async.bulk) into shared memory, with an mbarrier --
__device__ inline uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}" "\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ inline float coord_of(const unsigned char* pts, uint32_t i, int stride, int d) {
  return *reinterpret_cast<const float*>(pts + (uint64_t)i * (uint32_t)stride + 4u * d);
}
#endif

// ---------------------------------------------------------------------------
// Sets (batched builds).  A single build is a batch of one set.  Per level l
// the sets that still have a sort to run (L_b - 1 > l) are "active"; their
// compacted arrays are concatenated in set order.
struct SetInfo {
  uint32_t off;  // first record of the set in the caller's array
  uint32_t n;    // records in the set
};

// Outputs of the last pass of a per-dimension rank sort.
struct RankOut {
  uint32_t* rank;    // rank[item] in this dimension (one array per dimension), or nullptr
  uint32_t* rows;    // rank rows rows[4*item + d], rows[4*item + 3] = item (k <= 3), or nullptr
  uint32_t* sorted;  // sorted[position] = item, or nullptr
  int d;             // this dimension
  __device__ void put(uint32_t item, uint32_t r, uint32_t pos) const {
    if (rank) rank[item] = r;
    if (rows) {
      rows[4u * item + d] = r;
      if (d == 0) rows[4u * item + 3] = item;
    }
    if (sorted) sorted[pos] = item;
  }
};

struct ActiveEntry {
  uint32_t set;   // index into the set table
  uint32_t base;  // start of this set's items in the level's concatenated array
  int32_t next;   // index of the same set in the next level's active list, -1 if it leaves
  uint32_t box0;  // first box slot of this set at this level (widest mode)
  uint32_t chunk0;  // first key-build chunk of this set (segmented levels)
  uint32_t cps;     // key-build chunks per subtree segment (segmented levels)
};

}  // namespace kdb
