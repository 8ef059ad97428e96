// kdb_tree.cu -- per-level kernels of the k-d tree build other than the sort.
#include <algorithm>

#include "kdb_launch.h"

namespace kdb {

namespace {

constexpr int kThreads = 256;

// first set whose range contains record i (sets sorted by offset)
__device__ inline uint32_t find_set(const SetInfo* sets, uint32_t nsets, uint32_t i) {
  uint32_t lo = 0, hi = nsets;  // invariant: answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sets[mid].off <= i) lo = mid; else hi = mid;
  }
  while (lo + 1 < nsets && sets[lo].off + sets[lo].n <= i) ++lo;  // skip empty sets
  return lo;
}

__device__ inline uint32_t find_active(const ActiveEntry* act, uint32_t nact, uint32_t j) {
  uint32_t lo = 0, hi = nact;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (act[mid].base <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// warp-aggregated shared-memory histogram increment
__device__ inline void hist_add(uint32_t* h, uint32_t bin, bool ok) {
  const uint32_t b = ok ? bin : 0xFFFFFFFFu;
  const uint32_t peers = __match_any_sync(0xffffffffu, b);
  const int lane = threadIdx.x & 31;
  if (ok && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(h + bin, (uint32_t)__popc(peers));
}

// Contiguous chunk of [0, total) for this block, a multiple of blockDim long.
__device__ inline void block_chunk(uint32_t total, uint32_t* b, uint32_t* e) {
  const uint64_t per = (((uint64_t)total + gridDim.x - 1) / gridDim.x + blockDim.x - 1) /
                       blockDim.x * blockDim.x;
  const uint64_t s = per * blockIdx.x;
  *b = (uint32_t)(s < total ? s : total);
  *e = (uint32_t)(s + per < total ? s + per : total);
}

__device__ inline int widest_of(const float* lo, const float* hi, int k) {
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

// ---------------------------------------------------------------------------
// Prepass: coordinate keys for the per-dimension rank sorts, their digit
// histograms, the NaN check and (widest mode) each set's scene box, which is
// the domain of the root (Sec. 6).  One read of every record.
__global__ void __launch_bounds__(kThreads) prepass_kernel(PrepassArgs a) {
  extern __shared__ uint32_t s_hist[];
  const int H = a.hist ? a.k * a.passes * kRadixBins : 0;
  for (int i = threadIdx.x; i < H; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  // the launch's records [r0, r1), split into one chunk per block
  const uint32_t r0 = a.end ? a.beg : 0u, r1 = a.end ? a.end : a.total;
  uint32_t beg, end;
  block_chunk(r1 - r0, &beg, &end);
  beg += r0;
  end += r0;
  uint32_t lo[kMaxK], hi[kMaxK];
  for (int d = 0; d < kMaxK; ++d) {
    lo[d] = 0xFFFFFFFFu;
    hi[d] = 0u;
  }
  bool nan = false;
  uint32_t cur = 0;
  bool have = false;
  if (beg < end && a.nsets > 1) cur = find_set(a.sets, a.nsets, beg + threadIdx.x < end ? beg + threadIdx.x : beg);
  for (uint32_t base = beg; base < end; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const bool ok = i < end;
    if (ok && a.nsets > 1) {
      uint32_t s = cur;
      while (s + 1 < a.nsets && a.sets[s].off + a.sets[s].n <= i) ++s;
      if (s != cur && have && a.bbox) {
        for (int d = 0; d < a.k; ++d) {
          atomicMin(a.bbox + cur * 2 * a.k + d, lo[d]);
          atomicMax(a.bbox + cur * 2 * a.k + a.k + d, hi[d]);
          lo[d] = 0xFFFFFFFFu;
          hi[d] = 0u;
        }
      }
      cur = s;
    }
    have = have || ok;
    const unsigned char* rec = a.pts + (uint64_t)i * (uint32_t)a.stride;
    uint32_t ek[3] = {0u, 0u, 0u};
    for (int d = 0; d < a.k; ++d) {
      uint32_t key = 0;
      if (ok) {
        const uint32_t bits = *reinterpret_cast<const uint32_t*>(rec + 4 * d);
        if (!a.ctype && (bits & 0x7FFFFFFFu) > 0x7F800000u) nan = true;
        key = coord_key(bits, a.ctype);
        if (d < 3) ek[d] = key;
        lo[d] = min(lo[d], key);
        hi[d] = max(hi[d], key);
        if (a.keys32) a.keys32[(uint64_t)d * a.kstride + i] = key;
        if (a.keys64) a.keys64[(uint64_t)d * a.kstride + i] = ((uint64_t)cur << 32) | key;
      }
      if (a.hist) {
        // low digits spread over many bins: plain shared atomics; the top
        // float digit and the set-id digits repeat within a warp, so those
        // are aggregated per warp first
        const uint64_t k64 = ((uint64_t)cur << 32) | key;
        for (int p = 0; p < a.passes; ++p) {
          uint32_t* h = s_hist + (d * a.passes + p) * kRadixBins;
          const uint32_t bin = (uint32_t)(k64 >> (8 * p)) & (kRadixBins - 1);
          if (p < 3) {
            if (ok) atomicAdd(h + bin, 1u);
          } else {
            hist_add(h, bin, ok);
          }
        }
      }
    }
    if (a.ents && ok) a.ents[i] = make_uint4(ek[0], ek[1], ek[2], i);
  }
  if (a.bbox) {
    // warp-combine when the whole warp ended in one set, else per thread
    const uint32_t tag = have ? cur : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, tag);
    const int lane = threadIdx.x & 31;
    for (int d = 0; d < a.k; ++d) {
      uint32_t l = lo[d], h = hi[d];
      if (peers == 0xffffffffu) {
        l = __reduce_min_sync(0xffffffffu, l);
        h = __reduce_max_sync(0xffffffffu, h);
        if (lane == 0 && have) {
          atomicMin(a.bbox + cur * 2 * a.k + d, l);
          atomicMax(a.bbox + cur * 2 * a.k + a.k + d, h);
        }
      } else if (have) {
        atomicMin(a.bbox + cur * 2 * a.k + d, l);
        atomicMax(a.bbox + cur * 2 * a.k + a.k + d, h);
      }
    }
  }
  if (nan) atomicOr(a.err, ERR_NAN);
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += blockDim.x)
    if (s_hist[i]) atomicAdd(a.hist + i, s_hist[i]);
}

// ---------------------------------------------------------------------------
// The same prepass for the presorted-list path of one set with records of at
// most 16 bytes (k <= 3, payload allowed): each thread takes groups of four consecutive
// records, read as SW 16-byte words (SW = stride / 4, the group starts on a
// 16-byte boundary), two groups in flight, and writes their four entries.
// Records outside whole groups (the range's ragged ends) are done one by one.
// BITS > 0: also counts every digit of BITS bits of every key into s_hist
// ([dimension * passes + pass][2^BITS]).
template <int SW, int BITS>
__device__ inline void prepass_record(const PrepassArgs& a, uint32_t i, const uint32_t* w, uint32_t* lo,
                                      uint32_t* hi, bool* nan, uint32_t* s_hist) {
  uint32_t ek[3] = {0u, 0u, 0u};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d >= a.k) break;
    const uint32_t bits = w[d];
    if (!a.ctype && (bits & 0x7FFFFFFFu) > 0x7F800000u) *nan = true;
    const uint32_t key = coord_key(bits, a.ctype);
    ek[d] = key;
    lo[d] = min(lo[d], key);
    hi[d] = max(hi[d], key);
    if constexpr (BITS > 0) {
      constexpr int P = rec_passes(BITS);
      constexpr uint32_t R = 1u << BITS;
#pragma unroll
      for (int p = 0; p < P; ++p) atomicAdd(&s_hist[(d * P + p) * R + ((key >> (BITS * p)) & (R - 1u))], 1u);
    }
  }
  a.ents[i] = make_uint4(ek[0], ek[1], ek[2], i);
}

template <int SW, int BITS>
__global__ void __launch_bounds__(kThreads) prepass_vec_kernel(PrepassArgs a) {
  constexpr int HP = BITS > 0 ? 3 * rec_passes(BITS) << BITS : 1;
  __shared__ uint32_t s_hist[HP];
  if constexpr (BITS > 0) {
    for (int i = threadIdx.x; i < HP; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
  }
  const uint32_t r0 = a.end ? a.beg : 0u, r1 = a.end ? a.end : a.total;
  const uint32_t g0 = (r0 + 3u) / 4u, g1 = r1 / 4u;  // whole groups inside [r0, r1)
  uint32_t lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0u, 0u, 0u};
  bool nan = false;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  const uint4* src = reinterpret_cast<const uint4*>(a.pts);
  for (uint32_t g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += 2u * nthreads) {
    const uint32_t g2 = g + nthreads;
    uint4 va[SW], vb[SW];
#pragma unroll
    for (int q = 0; q < SW; ++q) va[q] = src[(uint64_t)g * SW + q];
    if (g2 < g1) {
#pragma unroll
      for (int q = 0; q < SW; ++q) vb[q] = src[(uint64_t)g2 * SW + q];
    }
    const uint32_t* wa = reinterpret_cast<const uint32_t*>(va);
#pragma unroll
    for (int j = 0; j < 4; ++j) prepass_record<SW, BITS>(a, 4u * g + j, wa + j * SW, lo, hi, &nan, s_hist);
    if (g2 < g1) {
      const uint32_t* wb = reinterpret_cast<const uint32_t*>(vb);
#pragma unroll
      for (int j = 0; j < 4; ++j) prepass_record<SW, BITS>(a, 4u * g2 + j, wb + j * SW, lo, hi, &nan, s_hist);
    }
  }
  // the ragged ends, by the first block
  if (blockIdx.x == 0) {
    const uint32_t h1 = min(4u * g0, r1), t0 = max(4u * g1, h1);
    for (uint32_t i = r0 + threadIdx.x; i < h1; i += blockDim.x) {
      uint32_t w[4];
      for (int d = 0; d < a.k; ++d) w[d] = reinterpret_cast<const uint32_t*>(a.pts)[(uint64_t)i * SW + d];
      prepass_record<SW, BITS>(a, i, w, lo, hi, &nan, s_hist);
    }
    for (uint32_t i = t0 + threadIdx.x; i < r1; i += blockDim.x) {
      uint32_t w[4];
      for (int d = 0; d < a.k; ++d) w[d] = reinterpret_cast<const uint32_t*>(a.pts)[(uint64_t)i * SW + d];
      prepass_record<SW, BITS>(a, i, w, lo, hi, &nan, s_hist);
    }
  }
  if (a.bbox) {
    const int lane = threadIdx.x & 31;
    for (int d = 0; d < a.k; ++d) {
      const uint32_t l = __reduce_min_sync(0xffffffffu, lo[d]);
      const uint32_t h = __reduce_max_sync(0xffffffffu, hi[d]);
      if (lane == 0 && l <= h) {
        atomicMin(a.bbox + d, l);
        atomicMax(a.bbox + a.k + d, h);
      }
    }
  }
  if (nan) atomicOr(a.err, ERR_NAN);
  if constexpr (BITS > 0) {
    __syncthreads();
    constexpr uint32_t R = 1u << BITS;
    const int H = a.k * rec_passes(BITS) * (int)R;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
      const uint32_t v = s_hist[i];
      if (v) atomicAdd(a.rec_hist + (uint32_t)i / R * kRadixBins + (uint32_t)i % R, v);
    }
  }
}

// ---------------------------------------------------------------------------
// Key of every item of level l: (active set, subtree, rank of the item in the
// subtree's split dimension).  The subtree of an item is implied by its
// position in the compacted array (Observation 3 / Sec. 4.2 inverted), so no
// tag is stored between levels.  Ranks order equal coordinates by original
// index, which makes the key strict.  Also builds the digit histograms of all
// passes of the level's sort.
__global__ void __launch_bounds__(kThreads) level_keys_kernel(LevelKeyArgs a) {
  __shared__ uint32_t s_hist[8 * kRadixBins];
  if (*reinterpret_cast<volatile uint32_t*>(a.x.err)) return;  // inputs may be garbage
  const int H = a.passes * kRadixBins;
  for (int i = threadIdx.x; i < H; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  uint32_t beg, end;
  block_chunk(a.items, &beg, &end);
  const LevelCtx& x = a.x;
  uint32_t ai = 0xFFFFFFFFu, aend = 0, abase = 0, soff = 0;
  LevelLayout y;
  const uint32_t Fl = full_nodes(x.l);
  for (uint32_t base = beg; base < end; base += blockDim.x) {
    const uint32_t j = base + threadIdx.x;
    const bool ok = j < end;
    uint64_t key = 0;
    if (ok) {
      if (ai == 0xFFFFFFFFu || j >= aend) {
        ai = (x.nact > 1) ? find_active(x.act, x.nact, j) : 0;
        const ActiveEntry e = x.act[ai];
        const SetInfo si = x.sets[e.set];
        y = LevelLayout::make(make_tree(si.n), x.l);
        abase = e.base;
        aend = e.base + y.items;
        soff = si.off;
      }
      const uint32_t jj = j - abase;
      const uint32_t s_rel = y.seg_of(jj);
      const uint32_t orig = a.vals ? a.vals[j] : soff + jj;
      if (!a.vals) a.vals_out[j] = orig;
      const int d = a.mode == 0 ? (x.l + x.dim0) % a.k : a.dims[soff + Fl + s_rel];
      uint32_t r = 0;
      if (orig < a.total && d < a.k) {
        r = a.ranks[(uint64_t)d * a.total + orig];
      } else {
        atomicOr(x.err, ERR_INTERNAL);
      }
      key = ((uint64_t)ai << (x.l + x.rb)) | ((uint64_t)s_rel << x.rb) | r;
      a.keys_out[j] = key;
    }
    for (int p = 0; p < a.passes; ++p)
      hist_add(s_hist + p * kRadixBins, (uint32_t)(key >> (8 * p)) & (kRadixBins - 1), ok);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += blockDim.x)
    if (s_hist[i]) atomicAdd(a.hist + i, s_hist[i]);
}

// Segmented variant: each block owns one chunk of one subtree segment, so the
// segment is known without a search and the block's digit histograms belong to
// one segment.  Key = rank of the item in its subtree's split dimension.
__global__ void __launch_bounds__(kThreads) seg_level_keys_kernel(SegKeyArgs a) {
  __shared__ uint32_t s_hist[4 * kRadixBins];
  if (*reinterpret_cast<volatile uint32_t*>(a.x.err)) return;
  const LevelCtx& x = a.x;
  const uint32_t g = blockIdx.x;
  uint32_t ai = 0;
  {
    uint32_t lo = 0, hi = x.nact;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (x.act[mid].chunk0 <= g) lo = mid; else hi = mid;
    }
    ai = lo;
  }
  const ActiveEntry e = x.act[ai];
  const SetInfo si = x.sets[e.set];
  const LevelLayout y = LevelLayout::make(make_tree(si.n), x.l);
  const uint32_t c = g - e.chunk0;
  const uint32_t s_rel = c / e.cps, ci = c % e.cps;
  if (s_rel >= y.nseg) return;
  const uint32_t sbeg = e.base + y.seg_start(s_rel), send = e.base + y.seg_start(s_rel + 1);
  const uint32_t beg = sbeg + ci * kSegChunk;
  if (beg >= send) return;
  const uint32_t end = beg + kSegChunk < send ? beg + kSegChunk : send;
  const int H = a.passes * kRadixBins;
  for (int i = threadIdx.x; i < H; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const int d = a.mode == 0 ? (x.l + x.dim0) % a.k : a.dims[si.off + full_nodes(x.l) + s_rel];
  const uint32_t* rank_d = a.ranks + (uint64_t)(d < a.k ? d : 0) * a.total;
  for (uint32_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
    const uint32_t orig = a.vals ? a.vals[j] : si.off + (j - e.base);
    if (!a.vals) a.vals_out[j] = orig;
    uint32_t r = 0;
    if (orig < a.total && d < a.k) r = rank_d[orig];
    else atomicOr(x.err, ERR_INTERNAL);
    a.keys_out[j] = r;
    for (int p = 0; p < a.passes; ++p) atomicAdd(&s_hist[p * kRadixBins + ((r >> (8 * p)) & 0xFF)], 1u);
  }
  __syncthreads();
  const uint32_t gid = (ai << x.l) | s_rel;
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    const uint32_t v = s_hist[i];
    if (v) {
      const int p = i / kRadixBins, dg = i % kRadixBins;
      atomicAdd(a.seg_hist + ((uint64_t)p * a.nseg + gid) * kRadixBins + dg, v);
    }
  }
}

// ---------------------------------------------------------------------------
// Split-widest (Sec. 6).  The domain of the root is the set's scene box; the
// domain of a child is its parent's domain with one side replaced by the
// parent's plane (hi = plane for the left child, lo = plane for the right
// child).  The paper recomputes a new subtree's domain by walking up to the
// root; here each level keeps the domains of its subtrees and derives the next
// level's from them, which yields the same boxes (a plane always lies inside
// its node's domain).  Split dimension = widest side (hi - lo in float32,
// first dimension wins ties).
__global__ void widest_root_kernel(const SetInfo* sets, const ActiveEntry* act, uint32_t nact,
                                   const uint32_t* bbox, int k, float* boxes, uint8_t* dims, int ctype) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nact) return;
  const ActiveEntry e = act[i];
  const uint32_t* lo = bbox + e.set * 2 * k;  // the scene box: the root's domain and its tight box
  const uint32_t* hi = lo + k;
  if (boxes)  // the root's domain, for the clipped-domain rule (float32 only)
    for (int d = 0; d < k; ++d) {
      boxes[(uint64_t)e.box0 * 2 * k + d] = __uint_as_float(key_to_float_bits(lo[d]));
      boxes[(uint64_t)e.box0 * 2 * k + k + d] = __uint_as_float(key_to_float_bits(hi[d]));
    }
  dims[sets[e.set].off] = (uint8_t)widest_of_keys(lo, hi, k, ctype);
}

__global__ void widest_children_kernel(WidestArgs a) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= a.total_threads) return;
  const LevelCtx& x = a.x;
  if (x.err && *reinterpret_cast<volatile uint32_t*>(x.err)) return;
  const uint32_t ei = tid >> x.l;
  const uint32_t s_rel = tid & ((1u << x.l) - 1u);
  const ActiveEntry e = x.act[ei];
  const SetInfo si = x.sets[e.set];
  const uint32_t s = full_nodes(x.l) + s_rel;
  const int k = a.k;
  float lo[kMaxK], hi[kMaxK];
  const float* bin = a.boxes_in + ((uint64_t)e.box0 + s_rel) * 2 * k;
  for (int d = 0; d < k; ++d) {
    lo[d] = bin[d];
    hi[d] = bin[k + d];
  }
  const int d = a.dims[si.off + s];
  const uint32_t node_rec = a.perm ? a.perm[si.off + s] : si.off + s;
  if (d >= k || node_rec >= si.off + si.n) {
    if (x.err) atomicOr(x.err, ERR_INTERNAL);
    return;
  }
  const float plane = coord_of(a.pts, node_rec, a.stride, d);
  const uint32_t c0 = 2 * s + 1;
  for (int side = 0; side < 2; ++side) {
    const uint32_t c = c0 + side;
    if (c >= si.n) break;
    const float keep = side == 0 ? hi[d] : lo[d];
    if (side == 0) hi[d] = plane; else lo[d] = plane;
    a.dims[si.off + c] = (uint8_t)widest_of(lo, hi, k);
    float* bout = nullptr;
    if (e.next >= 0)
      bout = a.boxes_out + ((uint64_t)x.act_next[e.next].box0 + 2 * s_rel + side) * 2 * k;
    else if (a.lsets)  // the child is the root of a subtree finished locally
      bout = a.boxes_local + ((uint64_t)a.lsets[e.set].lbox0 + 2 * s_rel + side) * 2 * k;
    if (bout) {
      for (int dd = 0; dd < k; ++dd) {
        bout[dd] = lo[dd];
        bout[k + dd] = hi[dd];
      }
    }
    if (side == 0) hi[d] = keep; else lo[d] = keep;
  }
}

__global__ void rr_dims_kernel(uint8_t* dims, const SetInfo* sets, uint32_t nsets, uint32_t total,
                               int k, int dim0) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const uint32_t s = nsets > 1 ? find_set(sets, nsets, i) : 0;
  dims[i] = (uint8_t)((level_of(i - sets[s].off) + dim0) % k);
}

// ---------------------------------------------------------------------------
// Final placement (Sec. 3.2: after the last iteration each point's tag is its
// node, and the array ends up sorted by tag), done as an almost-in-place
// permutation of the caller's records: perm[node] = original index is the one
// int32 per point; the staging area holds one record per kPermGroup nodes.
//
// perm splits into cycles.  Every block of kPermGroup consecutive nodes designates one
// "leader" (a hashed offset inside the block).  Phase 1 copies each leader's
// record aside.  Phase 2 starts one walker per leader: it fills its node from
// the node perm points to, moves there, and repeats until the next node is a
// leader, whose saved copy it takes.  Each node is written by exactly one
// walker, after that walker read it, so walkers never race.  A second round
// with denser leaders, then a minimum-index rotation, finish cycles that had
// no leader.  Visited nodes are marked in perm's top bit.
__device__ inline uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

__device__ inline uint32_t leader_of_block(uint32_t b, int round, uint32_t group) {
  return b * group + hash32(b ^ (0x9E3779B9u * (uint32_t)(round + 1))) % group;
}

__device__ inline bool is_leader(uint32_t node, int round, uint32_t group) {
  return leader_of_block(node / group, round, group) == node;
}

__device__ inline void copy_record(unsigned char* dst, const unsigned char* src, int stride) {
  if ((stride & 15) == 0 && ((((uintptr_t)dst) | ((uintptr_t)src)) & 15) == 0) {
    for (int o = 0; o < stride; o += 16)
      *reinterpret_cast<uint4*>(dst + o) = *reinterpret_cast<const uint4*>(src + o);
  } else {
    for (int o = 0; o < stride; o += 4)
      *reinterpret_cast<uint32_t*>(dst + o) = *reinterpret_cast<const uint32_t*>(src + o);
  }
}

__global__ void perm_stage_kernel(PermuteArgs a, int round, uint32_t group) {
  if (*a.err) return;
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nb = (a.total + group - 1) / group;
  if (b >= nb) return;
  const uint32_t ld = leader_of_block(b, round, group);
  if (ld >= a.total || (a.perm[ld] & kMark)) return;
  copy_record(a.stage + (uint64_t)b * a.stride, a.pts + (uint64_t)ld * a.stride, a.stride);
}

__global__ void perm_walk_kernel(PermuteArgs a, int round, uint32_t group) {
  if (*a.err) return;
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nb = (a.total + group - 1) / group;
  if (b >= nb) return;
  const uint32_t ld = leader_of_block(b, round, group);
  if (ld >= a.total || (a.perm[ld] & kMark)) return;
  uint32_t cur = ld;
  uint32_t nxt = a.perm[cur] & ~kMark;
  for (uint32_t steps = 0; steps <= a.total; ++steps) {
    if (nxt >= a.total) {
      atomicOr(a.err, ERR_INTERNAL);
      return;
    }
    unsigned char* dst = a.pts + (uint64_t)cur * a.stride;
    if (is_leader(nxt, round, group)) {
      copy_record(dst, a.stage + (uint64_t)(nxt / group) * a.stride, a.stride);
      a.perm[cur] = nxt | kMark;
      return;
    }
    // the next link is read together with the record, so a step costs one
    // memory latency, not two
    const uint32_t after = a.perm[nxt] & ~kMark;
    copy_record(dst, a.pts + (uint64_t)nxt * a.stride, a.stride);
    a.perm[cur] = nxt | kMark;
    cur = nxt;
    nxt = after;
  }
  atomicOr(a.err, ERR_INTERNAL);  // longer than any cycle: perm is not a permutation
}

__global__ void perm_rest_kernel(PermuteArgs a) {
  if (*a.err) return;
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.total) return;
  if (a.perm[s] & kMark) return;
  // the rotation is done by the smallest node of the cycle
  uint32_t x = a.perm[s] & ~kMark;
  for (uint32_t steps = 0; x != s; ++steps) {
    if (x < s) return;
    if (steps > a.total || x >= a.total) {
      atomicOr(a.err, ERR_INTERNAL);
      return;
    }
    x = a.perm[x] & ~kMark;
  }
  uint4 tmp4[16];
  unsigned char* tmp = reinterpret_cast<unsigned char*>(tmp4);
  const bool small = a.stride <= 256;
  uint32_t cur = s;
  if (small) copy_record(tmp, a.pts + (uint64_t)s * a.stride, a.stride);
  // records longer than 256 bytes rotate the other way round: swap along the cycle
  for (;;) {
    const uint32_t nxt = a.perm[cur] & ~kMark;
    if (nxt == s) {
      if (small) copy_record(a.pts + (uint64_t)cur * a.stride, tmp, a.stride);
      a.perm[cur] |= kMark;
      return;
    }
    if (small) {
      copy_record(a.pts + (uint64_t)cur * a.stride, a.pts + (uint64_t)nxt * a.stride, a.stride);
    } else {
      uint32_t* p = reinterpret_cast<uint32_t*>(a.pts + (uint64_t)cur * a.stride);
      uint32_t* q = reinterpret_cast<uint32_t*>(a.pts + (uint64_t)nxt * a.stride);
      for (int o = 0; o < a.stride / 4; ++o) {
        const uint32_t t = p[o];
        p[o] = q[o];
        q[o] = t;
      }
    }
    a.perm[cur] |= kMark;
    cur = nxt;
  }
}

// Placement through spare workspace: tmp[i] = record of node i (its original
// position perm[i]), then one coalesced copy back.  Same result as the cycle
// walk; used when the workspace that is dead by now can hold the records.
constexpr int kGatherStage = 64;  // records up to this stride are staged per block
__global__ void __launch_bounds__(kThreads) place_gather_kernel(PermuteArgs a, unsigned char* tmp) {
  __shared__ __align__(16) uint32_t s_rec[kThreads * kGatherStage / 4];
  if (*reinterpret_cast<volatile uint32_t*>(a.err)) return;
  const uint32_t i0 = blockIdx.x * kThreads;
  const uint32_t i = i0 + threadIdx.x;
  const int words = a.stride / 4;
  uint32_t src = 0;
  bool ok = i < a.total;
  if (ok) {
    src = a.perm[i] & ~kMark;
    if (src >= a.total) {
      atomicOr(a.err, ERR_INTERNAL);
      ok = false;
    }
  }
  if (a.stride > kGatherStage) {
    if (ok) copy_record(tmp + (uint64_t)i * a.stride, a.pts + (uint64_t)src * a.stride, a.stride);
    return;
  }
  if (ok) {
    const uint32_t* r = reinterpret_cast<const uint32_t*>(a.pts + (uint64_t)src * a.stride);
    for (int w = 0; w < words; ++w) s_rec[threadIdx.x * words + w] = r[w];
  }
  __syncthreads();
  // the block's records are contiguous in tmp: write them word by word
  const uint32_t n = min((uint32_t)kThreads, a.total - i0);
  uint32_t* out = reinterpret_cast<uint32_t*>(tmp + (uint64_t)i0 * a.stride);
  for (uint32_t w = threadIdx.x; w < n * (uint32_t)words; w += kThreads) out[w] = s_rec[w];
}

__global__ void place_copy_back_kernel(PermuteArgs a, const unsigned char* tmp, uint64_t bytes) {
  if (*reinterpret_cast<volatile uint32_t*>(a.err)) return;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (((reinterpret_cast<uintptr_t>(a.pts) | reinterpret_cast<uintptr_t>(tmp) | bytes) & 15) == 0) {
    const uint4* s = reinterpret_cast<const uint4*>(tmp);
    uint4* d = reinterpret_cast<uint4*>(a.pts);
    for (uint64_t q = t0; q < bytes / 16; q += stride) d[q] = s[q];
  } else {
    const uint32_t* s = reinterpret_cast<const uint32_t*>(tmp);
    uint32_t* d = reinterpret_cast<uint32_t*>(a.pts);
    for (uint64_t q = t0; q < bytes / 4; q += stride) d[q] = s[q];
  }
}

// After a failed build that wrote records at their nodes: put every record
// back from its entry, so the caller's array is as it was.
__global__ void restore_kernel(unsigned char* pts, const uint4* ents, uint32_t total, int k,
                               const uint32_t* err, int ctype) {
  if (*reinterpret_cast<const volatile uint32_t*>(err) == 0) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
    write_record_from_entry(pts + (uint64_t)i * (4 * k), ents[i], k, ctype);
}

// Scene-box accumulators of every set: lower keys at the top, upper at zero.
__global__ void init_bbox_kernel(uint32_t* bbox, uint32_t nsets, int k) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsets * 2 * (uint32_t)k) return;
  bbox[i] = (i % (2 * (uint32_t)k)) < (uint32_t)k ? 0xFFFFFFFFu : 0u;
}

__global__ void unmark_kernel(const uint32_t* perm, int32_t* out, uint32_t total) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) out[i] = (int32_t)(perm[i] & ~kMark);
}

// ---------------------------------------------------------------------------
// k-d condition of every node against every ancestor (Sec. 1), in the total
// order of float_key (-0 < +0); ties are allowed on both sides.
// Tight-box rule in the validator: the box of node i's subtree is its own
// point joined with its children's boxes, built bottom-up one level per launch
// (keys, so that min / max follow the strict order); the node's dimension is
// the widest side of that box.
__global__ void tight_box_level_kernel(const unsigned char* pts, uint32_t n, int k, int stride, int l,
                                       uint32_t* box, uint8_t* dims, int ctype) {
  const uint64_t i = (uint64_t)full_nodes(l) + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n || i >= (uint64_t)full_nodes(l + 1)) return;
  uint32_t lo[kMaxK], hi[kMaxK];
  for (int d = 0; d < k; ++d)
    lo[d] = hi[d] = coord_key(__float_as_uint(coord_of(pts, (uint32_t)i, stride, d)), ctype);
  for (uint64_t c = 2 * i + 1; c <= 2 * i + 2 && c < n; ++c)
    for (int d = 0; d < k; ++d) {
      lo[d] = min(lo[d], box[c * 2 * k + d]);
      hi[d] = max(hi[d], box[c * 2 * k + k + d]);
    }
  for (int d = 0; d < k; ++d) {
    box[i * 2 * k + d] = lo[d];
    box[i * 2 * k + k + d] = hi[d];
  }
  dims[i] = (uint8_t)widest_of_keys(lo, hi, k, ctype);
}

__global__ void validate_kernel(const unsigned char* pts, uint32_t n, int k, int stride, int mode,
                                const uint8_t* dims, uint32_t* first_bad) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 || i >= n) return;
  uint32_t child = i;
  uint32_t p = (i - 1) / 2;
  const int ctype = (mode & 0x100) ? kCoordI32 : ((mode & 0x200) ? kCoordU32 : kCoordF32);
  for (;;) {
    const int d = (mode & 0xFF) == 0 ? level_of(p) % k : dims[p];
    const uint32_t ki = coord_key(__float_as_uint(coord_of(pts, i, stride, d)), ctype);
    const uint32_t kp = coord_key(__float_as_uint(coord_of(pts, p, stride, d)), ctype);
    const bool left = child == 2 * p + 1;
    if ((left && ki > kp) || (!left && ki < kp)) {
      atomicMin(first_bad, i);
      return;
    }
    if (p == 0) return;
    child = p;
    p = (p - 1) / 2;
  }
}

}  // namespace

// ------------------------------------------------------------- launchers --
// one set, entries only, records of 4k <= 16 bytes on a 16-byte boundary:
// the vectorised prepass
bool prepass_fuses_rec_hist(const PrepassArgs& a) {
  return a.ents && !a.hist && !a.keys32 && !a.keys64 && a.nsets == 1 && a.k <= 3 && a.stride <= 16 &&
         a.stride % 4 == 0 && 4 * a.k <= a.stride && (reinterpret_cast<uintptr_t>(a.pts) & 15u) == 0;
}

template <int BITS>
void launch_prepass_vec(const PrepassArgs& a, uint32_t grid, cudaStream_t st) {
  switch (a.stride / 4) {
    case 1: prepass_vec_kernel<1, BITS><<<grid, kThreads, 0, st>>>(a); break;
    case 2: prepass_vec_kernel<2, BITS><<<grid, kThreads, 0, st>>>(a); break;
    case 3: prepass_vec_kernel<3, BITS><<<grid, kThreads, 0, st>>>(a); break;
    default: prepass_vec_kernel<4, BITS><<<grid, kThreads, 0, st>>>(a); break;
  }
}

cudaError_t launch_prepass(const PrepassArgs& a, int num_sms, cudaStream_t st) {
  const uint32_t count = a.end ? a.end - a.beg : a.total;
  if (count == 0) return cudaSuccess;
  if (prepass_fuses_rec_hist(a)) {
    uint32_t grid = (uint32_t)num_sms * 8;
    const uint32_t need = (count / 4 + 2 * kThreads - 1) / (2 * kThreads);
    if (grid > need) grid = need > 0 ? need : 1;
    static_assert(kRecDigitWidths == 2, "one launcher per width");
    if (!a.rec_hist) launch_prepass_vec<0>(a, grid, st);
    else if (a.rec_bits == 6) launch_prepass_vec<6>(a, grid, st);
    else launch_prepass_vec<8>(a, grid, st);
    return cudaGetLastError();
  }
  const size_t smem = a.hist ? (size_t)a.k * a.passes * kRadixBins * sizeof(uint32_t) : 0;
  cudaError_t e = ensure_smem((const void*)prepass_kernel, smem);
  if (e != cudaSuccess) return e;
  uint32_t grid = (uint32_t)num_sms * 4;
  const uint32_t need = (count + kThreads - 1) / kThreads;
  if (grid > need) grid = need;
  prepass_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_level_keys(const LevelKeyArgs& a, int num_sms, cudaStream_t st) {
  if (a.items == 0) return cudaSuccess;
  uint32_t grid = (uint32_t)num_sms * 8;
  const uint32_t need = (a.items + kThreads - 1) / kThreads;
  if (grid > need) grid = need;
  level_keys_kernel<<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_seg_level_keys(const SegKeyArgs& a, cudaStream_t st) {
  if (a.chunks == 0) return cudaSuccess;
  seg_level_keys_kernel<<<a.chunks, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_widest_root(const SetInfo* sets, const ActiveEntry* act0, uint32_t nact,
                               const uint32_t* bbox, int k, float* boxes0, uint8_t* dims, int ctype,
                               cudaStream_t st) {
  if (nact == 0) return cudaSuccess;
  widest_root_kernel<<<(nact + 127) / 128, 128, 0, st>>>(sets, act0, nact, bbox, k, boxes0, dims, ctype);
  return cudaGetLastError();
}

cudaError_t launch_tight_validate_dims(const unsigned char* pts, uint32_t n, int k, int stride,
                                       uint32_t* box, uint8_t* dims, int ctype, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  for (int l = num_levels(n) - 1; l >= 0; --l) {
    const uint32_t cnt = std::min<uint64_t>((uint64_t)n, (uint64_t)full_nodes(l + 1)) - full_nodes(l);
    tight_box_level_kernel<<<(cnt + kThreads - 1) / kThreads, kThreads, 0, st>>>(pts, n, k, stride, l,
                                                                                   box, dims, ctype);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_widest_children(const WidestArgs& a, cudaStream_t st) {
  if (a.total_threads == 0) return cudaSuccess;
  widest_children_kernel<<<(a.total_threads + kThreads - 1) / kThreads, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rr_dims(uint8_t* dims, const SetInfo* sets, uint32_t nsets, uint32_t total,
                           int k, int dim0, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  rr_dims_kernel<<<(total + kThreads - 1) / kThreads, kThreads, 0, st>>>(dims, sets, nsets, total, k,
                                                                          dim0);
  return cudaGetLastError();
}

cudaError_t launch_permute(const PermuteArgs& a, int num_sms, cudaStream_t st) {
  (void)num_sms;
  if (a.total == 0) return cudaSuccess;
  // both rounds use one leader per kPermGroup nodes (the staging area holds
  // ceil(total / kPermGroup) records); the second round hashes to other offsets
  const uint32_t groups[2] = {kPermGroup, kPermGroup};
  for (int r = 0; r < 2; ++r) {
    const uint32_t nb = (a.total + groups[r] - 1) / groups[r];
    const uint32_t grid = (nb + kThreads - 1) / kThreads;
    perm_stage_kernel<<<grid, kThreads, 0, st>>>(a, r, groups[r]);
    perm_walk_kernel<<<grid, kThreads, 0, st>>>(a, r, groups[r]);
  }
  perm_rest_kernel<<<(a.total + kThreads - 1) / kThreads, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_place_gather(const PermuteArgs& a, unsigned char* tmp, int num_sms, cudaStream_t st) {
  if (a.total == 0) return cudaSuccess;
  place_gather_kernel<<<(a.total + kThreads - 1) / kThreads, kThreads, 0, st>>>(a, tmp);
  const uint64_t bytes = (uint64_t)a.total * a.stride;
  const uint64_t want = (bytes / 16 + kThreads - 1) / kThreads;
  const uint32_t grid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(want, 1), (uint64_t)num_sms * 8);
  place_copy_back_kernel<<<grid, kThreads, 0, st>>>(a, tmp, bytes);
  return cudaGetLastError();
}

cudaError_t launch_restore(unsigned char* pts, const uint4* ents, uint32_t total, int k, const uint32_t* err,
                           int ctype, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  // a small grid: the kernel usually finds no error and returns at once
  const uint32_t grid = std::min<uint32_t>((total + kThreads - 1) / kThreads, 1024);
  restore_kernel<<<grid, kThreads, 0, st>>>(pts, ents, total, k, err, ctype);
  return cudaGetLastError();
}

cudaError_t launch_init_bbox(uint32_t* bbox, uint32_t nsets, int k, cudaStream_t st) {
  const uint32_t n = nsets * 2 * (uint32_t)k;
  if (n == 0) return cudaSuccess;
  init_bbox_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(bbox, nsets, k);
  return cudaGetLastError();
}

cudaError_t launch_unmark(const uint32_t* perm, int32_t* out, uint32_t total, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  unmark_kernel<<<(total + kThreads - 1) / kThreads, kThreads, 0, st>>>(perm, out, total);
  return cudaGetLastError();
}

cudaError_t launch_validate(const unsigned char* pts, uint32_t n, int k, int stride, int mode,
                            const uint8_t* dims, uint32_t* first_bad, cudaStream_t st) {
  if (n < 2) return cudaSuccess;
  validate_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(pts, n, k, stride, mode, dims,
                                                                        first_bad);
  return cudaGetLastError();
}

}  // namespace kdb
