// kdb_segsort.cuh -- segmented onesweep radix pass (32-bit keys).
//
// After the fused tag update of level l-1 the live items of level l are
// already grouped by subtree, each subtree's items contiguous and in subtree
// order (Observation 3).  The level-l sort by (tag, coordinate) (Sec. 3.1)
// therefore only has to order every segment by its items' ranks: the tag is
// never part of the key.  This pass sorts each segment independently by one
// 8-bit digit of the 32-bit key, stably, with per-(segment, digit) bins.
//
// Requirement: every segment of the level is at least one tile long, so a
// tile holds the tail of one segment (A) and possibly the head of the next
// (B).  Only A can continue from earlier tiles; the look-back words of a
// tile always describe its last segment, and a tile whose last segment starts
// inside it publishes an inclusive prefix at once.
#pragma once

#include "kdb_launch.h"
#include "kdb_onesweep.cuh"

namespace kdb {

// Where the tile's (at most two) segments are.
struct TileSegs {
  uint32_t ai[2];     // active entry of segment A / B
  uint32_t srel[2];   // subtree index within its set's level
  uint32_t start[2];  // first position of the segment in the level array
  uint32_t gid[2];    // global segment id: (ai << l) | srel
  uint32_t bpos;      // tile position where B begins (== tile length if none)
  // for the fused tag update
  uint32_t pr[2];     // pivot rank ss(lChild(s)) (Observation 1)
  uint32_t ebase[2];  // first position of the segment's set in this level
  uint32_t node[2];   // first slot of the set in perm + F(l) + srel: node s
  uint32_t child0[2]; // where the set's children go: next level's base, the
                      // set's first record (local level array), or its
                      // lowest-level slot F(l+1) in perm
  int32_t next[2];    // 0: next level's array, 1: perm (lowest level), 2: local array
};

__device__ inline void fill_update_info(const LevelCtx& x, TileSegs& ts, int i) {
  const ActiveEntry e = x.act[ts.ai[i]];
  const SetInfo si = x.sets[e.set];
  const LevelLayout y = LevelLayout::make(make_tree(si.n), x.l);
  ts.pr[i] = y.left_size(ts.srel[i]);
  ts.ebase[i] = e.base;
  ts.node[i] = si.off + full_nodes(x.l) + ts.srel[i];
  if (e.next >= 0) {
    ts.next[i] = 0;
    ts.child0[i] = x.act_next[e.next].base;
  } else if (x.local_next) {
    ts.next[i] = 2;
    ts.child0[i] = si.off;
  } else {
    ts.next[i] = 1;
    ts.child0[i] = si.off + full_nodes(x.l + 1);
  }
}

__device__ inline uint32_t find_active_entry(const ActiveEntry* act, uint32_t nact, uint32_t j) {
  uint32_t lo = 0, hi = nact;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (act[mid].base <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// Segment containing position j of level x.l, with its bounds.
__device__ inline void segment_at(const LevelCtx& x, uint32_t j, uint32_t* ai, uint32_t* srel,
                                  uint32_t* start, uint32_t* end) {
  const uint32_t a = x.nact > 1 ? find_active_entry(x.act, x.nact, j) : 0;
  const ActiveEntry e = x.act[a];
  const LevelLayout y = LevelLayout::make(make_tree(x.sets[e.set].n), x.l);
  const uint32_t s = y.seg_of(j - e.base);
  *ai = a;
  *srel = s;
  *start = e.base + y.seg_start(s);
  *end = e.base + y.seg_start(s + 1);
}

template <int THREADS, int ITEMS, class Epi>
__global__ void __launch_bounds__(THREADS)
    seg_onesweep_pass(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                      PassCtl c, LevelCtx x, const uint32_t* __restrict__ seg_hist, Epi epi) {
  static_assert(THREADS == kRadix, "one thread per digit");
  constexpr int WARPS = THREADS / 32;
  constexpr int TILE = THREADS * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* s_vals = s_keys + TILE;
  __shared__ uint32_t s_whist[WARPS][2 * kRadix];
  __shared__ uint32_t s_gbase[2 * kRadix];
  __shared__ uint32_t s_toff[2 * kRadix];  // tile offset of each bin (A bins, then B bins)
  __shared__ uint32_t s_toffB0;  // first staged position of segment B
  __shared__ uint32_t s_scan[WARPS];
  __shared__ uint32_t s_tile, s_abort;
  __shared__ TileSegs s_ts;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_abort = *reinterpret_cast<volatile uint32_t*>(c.err) != 0u;
    if (!s_abort) {
      const uint32_t tile = atomicAdd(c.ticket, 1u);
      s_tile = tile;
      const uint32_t tb = tile * (uint32_t)TILE;
      const uint32_t tn = c.n - tb < (uint32_t)TILE ? c.n - tb : (uint32_t)TILE;
      uint32_t a, s, st, en;
      segment_at(x, tb, &a, &s, &st, &en);
      s_ts.ai[0] = a;
      s_ts.srel[0] = s;
      s_ts.start[0] = st;
      s_ts.gid[0] = (a << x.l) | s;
      s_ts.bpos = tn;
      if (en < tb + tn) {  // the tile reaches into the next segment
        uint32_t a2, s2, st2, en2;
        segment_at(x, en, &a2, &s2, &st2, &en2);
        s_ts.ai[1] = a2;
        s_ts.srel[1] = s2;
        s_ts.start[1] = st2;
        s_ts.gid[1] = (a2 << x.l) | s2;
        s_ts.bpos = en - tb;
        if (en2 < tb + tn) s_abort = 2;  // a segment shorter than a tile: not allowed here
      } else {
        s_ts.ai[1] = a;
        s_ts.srel[1] = s;
        s_ts.start[1] = st;
        s_ts.gid[1] = s_ts.gid[0];
      }
      if (Epi::kNeedsUpdateInfo) {
        fill_update_info(x, s_ts, 0);
        fill_update_info(x, s_ts, 1);
      }
    }
  }
  for (int i = tid; i < WARPS * 2 * kRadix; i += THREADS) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  if (s_abort == 1) return;
  if (s_abort == 2) {
    // cannot happen with the level plan; record it and publish so no tile waits
    if (tid == 0) atomicOr(c.err, ERR_INTERNAL);
  }
  const uint32_t tile = s_tile;
  const uint32_t tb = tile * (uint32_t)TILE;
  const uint32_t tn = c.n - tb < (uint32_t)TILE ? c.n - tb : (uint32_t)TILE;
  const uint32_t bpos = s_ts.bpos;
  const bool hasB = bpos < tn;
  const bool a_cont = s_ts.start[0] < tb;  // segment A began in an earlier tile
  const uint32_t wbase = (uint32_t)warp * 32 * ITEMS;

  uint32_t key[ITEMS], val[ITEMS], rnk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    if (p < tn) {
      key[i] = keys_in[tb + p];
      val[i] = vals_in[tb + p];
    }
  }
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    const bool ok = p < tn;
    const uint32_t bin =
        ok ? (((p >= bpos) ? (uint32_t)kRadix : 0u) | digit_of(key[i], c.shift)) : 2u * kRadix;
    const uint32_t peers = __match_any_sync(0xffffffffu, bin);
    uint32_t before = 0;
    if (ok) before = s_whist[warp][bin];
    __syncwarp();
    if (ok) {
      rnk[i] = before + __popc(peers & lt);
      if ((peers & lt) == 0) s_whist[warp][bin] = before + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();

  // per bin (thread tid owns digit tid of A and of B)
  uint32_t cA = 0, cB = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    const uint32_t ta = s_whist[w][tid], tb2 = s_whist[w][kRadix + tid];
    s_whist[w][tid] = cA;
    s_whist[w][kRadix + tid] = cB;
    cA += ta;
    cB += tb2;
  }
  uint32_t totA, totB, d0;
  const uint32_t toffA = block_excl_scan<THREADS>(cA, s_scan, &totA);
  const uint32_t toffB = block_excl_scan<THREADS>(cB, s_scan, &totB) + totA;
  const uint32_t hA = seg_hist[(uint64_t)s_ts.gid[0] * kRadix + tid];
  const uint32_t hB = hasB ? seg_hist[(uint64_t)s_ts.gid[1] * kRadix + tid] : 0u;
  const uint32_t bA = block_excl_scan<THREADS>(hA, s_scan, &d0);
  const uint32_t bB = block_excl_scan<THREADS>(hB, s_scan, &d0);

  // look-back for segment A's digit prefixes; publish for the tile's last segment
  uint64_t* mine = c.status + (uint64_t)tile * kRadix + tid;
  uint32_t prefA = 0;
  if (hasB || !a_cont) st_relaxed_u64(mine, lb_pack(kFlagPre, c.epoch, hasB ? cB : cA));
  else st_relaxed_u64(mine, lb_pack(kFlagAgg, c.epoch, cA));
  if (a_cont && s_abort == 0) {
    int64_t t = (int64_t)tile - 1;
    bool waiting = false, expired = false;
    uint64_t t0 = 0;
    for (;;) {
      const uint64_t w = ld_relaxed_u64(c.status + (uint64_t)t * kRadix + tid);
      const uint32_t ep = (uint32_t)(w >> 32) & 0x3FFFFFFFu;
      if (ep == c.wait_epoch && (w >> 62) != 0) {
        prefA += (uint32_t)w;
        if ((w >> 62) == 2 || t == 0) break;
        --t;
        waiting = false;
        continue;
      }
      const uint64_t now = global_timer_ns();
      if (!waiting) {
        waiting = true;
        t0 = now;
      } else if (now - t0 > c.wait_ns) {
        expired = true;
        break;
      }
    }
    if (expired) {
      atomicOr(c.err, ERR_TIMEOUT);
      s_abort = 1;
    }
    if (!hasB) st_relaxed_u64(mine, lb_pack(kFlagPre, c.epoch, prefA + cA));
  }
  s_toff[tid] = toffA;
  s_toff[kRadix + tid] = toffB;
  s_gbase[tid] = s_ts.start[0] + bA + prefA - toffA;
  s_gbase[kRadix + tid] = s_ts.start[1] + bB - toffB;
  if (tid == 0) s_toffB0 = totA;
  __syncthreads();
  if (s_abort) return;

#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    if (p < tn) {
      const uint32_t bin = ((p >= bpos) ? (uint32_t)kRadix : 0u) | digit_of(key[i], c.shift);
      const uint32_t pos = s_toff[bin] + s_whist[warp][bin] + rnk[i];
      s_keys[pos] = key[i];
      s_vals[pos] = val[i];
    }
  }
  __syncthreads();
  for (uint32_t p = tid; p < tn; p += THREADS) {
    const uint32_t k = s_keys[p];
    const uint32_t seg = p >= s_toffB0 ? 1u : 0u;
    const uint32_t bin = (seg ? (uint32_t)kRadix : 0u) | digit_of(k, c.shift);
    const uint32_t dest = s_gbase[bin] + p;
    if (dest >= c.n) {
      atomicOr(c.err, ERR_INTERNAL);
      continue;
    }
    epi(k, s_vals[p], dest, seg, s_ts);
  }
}

// ---- epilogues ------------------------------------------------------------
struct SegEpiPingPong {
  static constexpr bool kNeedsUpdateInfo = false;
  uint32_t* keys_out;
  uint32_t* vals_out;
  __device__ void operator()(uint32_t k, uint32_t v, uint32_t dest, uint32_t, const TileSegs&) const {
    keys_out[dest] = k;
    vals_out[dest] = v;
  }
};

// Tag update of Sec. 3.2 on the level's last pass: `dest` is the item's
// position in the sorted level array, so its rank inside its subtree's
// segment is q = dest - sb(s) (Sec. 4.2).  q == ss(lChild(s)) pins the item as
// node s; smaller q go to lChild(s), larger to rChild(s), written straight
// into the next level's compacted array (one pinned item removed per earlier
// subtree, plus this subtree's own pivot for right children).  On a set's last
// sorted level the children are lowest-level nodes and go to their slots.
struct SegEpiUpdate {
  static constexpr bool kNeedsUpdateInfo = true;
  uint32_t* perm;
  uint32_t* vals_next;
  uint32_t* vals_local;
  __device__ void operator()(uint32_t, uint32_t orig, uint32_t dest, uint32_t seg,
                             const TileSegs& ts) const {
    const uint32_t q = dest - ts.start[seg];
    const uint32_t pr = ts.pr[seg];
    if (q == pr) {
      perm[ts.node[seg]] = orig;
      return;
    }
    const uint32_t jn = dest - ts.ebase[seg] - ts.srel[seg] - (q > pr ? 1u : 0u);
    uint32_t* out = ts.next[seg] == 0 ? vals_next : (ts.next[seg] == 1 ? perm : vals_local);
    out[ts.child0[seg] + jn] = orig;
  }
};

}  // namespace kdb
