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

// Exclusive block scan of one 64-bit value per thread (any multiple of 32
// threads up to 1024).
template <int THREADS>
__device__ inline uint64_t block_excl_scan64(uint64_t v, uint64_t* s_tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < THREADS / 32 ? s_tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < THREADS / 32) s_tmp[lane] = w;
  }
  __syncthreads();
  const uint64_t r = (warp ? s_tmp[warp - 1] : 0) + x - v;
  __syncthreads();
  return r;
}

// Bound on waiting for the tile's bulk copy; after it the block records a
// timeout, waits the same again for the copy to land, and leaves.
constexpr uint64_t kCopyWaitNs = 2000000000ull;

template <int THREADS, int ITEMS, int MINB, class Epi>
__global__ void __launch_bounds__(THREADS, MINB)
    seg_onesweep_pass(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                      PassCtl c, LevelCtx x, const uint32_t* __restrict__ seg_hist, Epi epi) {
  static_assert(THREADS >= kRadix && THREADS % 32 == 0, "a thread per digit");
  static_assert((THREADS * ITEMS) % 4 == 0, "tiles start on 16-byte boundaries");
  constexpr int WARPS = THREADS / 32;
  constexpr int TILE = THREADS * ITEMS;
  constexpr int BINS = 2 * kRadix;  // (segment A or B) x digit
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(smem_raw);          // tile in, then out
  uint32_t* s_vals = s_keys + TILE;                                   // tile in, then out
  uint16_t* s_whist = reinterpret_cast<uint16_t*>(s_vals + TILE);     // [BINS][WARPS]
  __shared__ uint32_t s_gbase[BINS];
  __shared__ uint32_t s_toff[BINS];
  __shared__ uint64_t s_scan64[WARPS];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile, s_abort, s_totA;
  __shared__ TileSegs s_ts;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_abort = *reinterpret_cast<volatile uint32_t*>(c.err) != 0u;
    if (!s_abort) {
      s_tile = atomicAdd(c.ticket, 1u);
      if ((uint64_t)(s_tile + 1) * kRadix > c.status_words) {  // the last tiles: no tile waits on them
        atomicOr(c.err, ERR_INTERNAL);
        s_abort = 1;
      }
    }
    if (!s_abort) {
      const uint32_t tile = s_tile;
      const uint32_t tb = tile * (uint32_t)TILE;
      const uint32_t tn = c.n - tb < (uint32_t)TILE ? c.n - tb : (uint32_t)TILE;
      // 1. the tile's keys and values to shared memory by bulk copy (whole
      //    16-byte groups; the last 0-3 items are loaded below)
      const uint32_t nal = tn & ~3u;
      mbar_init(&s_bar, 1);
      mbar_expect_tx(&s_bar, nal * 4u * (vals_in ? 2u : 1u));
      if (nal) {
        bulk_g2s(s_keys, keys_in + tb, nal * 4u, &s_bar);
        if (vals_in) bulk_g2s(s_vals, vals_in + tb, nal * 4u, &s_bar);
      }
      uint32_t a, sr, st, en;
      segment_at(x, tb, &a, &sr, &st, &en);
      s_ts.ai[0] = a;
      s_ts.srel[0] = sr;
      s_ts.start[0] = st;
      s_ts.gid[0] = (a << x.l) | sr;
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
        s_ts.srel[1] = sr;
        s_ts.start[1] = st;
        s_ts.gid[1] = s_ts.gid[0];
      }
      if (Epi::kNeedsUpdateInfo) {
        fill_update_info(x, s_ts, 0);
        fill_update_info(x, s_ts, 1);
      }
    }
  }
  for (int i = tid; i < BINS * WARPS / 2; i += THREADS) reinterpret_cast<uint32_t*>(s_whist)[i] = 0;
  __syncthreads();
  if (s_abort == 1) return;
  if (s_abort == 2 && tid == 0) atomicOr(c.err, ERR_INTERNAL);
  const uint32_t tile = s_tile;
  const uint32_t tb = tile * (uint32_t)TILE;
  const uint32_t tn = c.n - tb < (uint32_t)TILE ? c.n - tb : (uint32_t)TILE;
  const uint32_t nal = tn & ~3u;
  if (tid < (int)(tn - nal)) {
    s_keys[nal + tid] = keys_in[tb + nal + tid];
    if (vals_in) s_vals[nal + tid] = vals_in[tb + nal + tid];
  }
  if (!vals_in)
    for (uint32_t p = tid; p < tn; p += THREADS) s_vals[p] = tb + p;
  {
    bool waiting = false, late = false;
    uint64_t t0 = 0;
    while (!mbar_try_wait(&s_bar, 0)) {
      const uint64_t now = global_timer_ns();
      if (!waiting) {
        waiting = true;
        t0 = now;
      } else if (now - t0 > (late ? 2 : 1) * kCopyWaitNs) {
        if (late) break;  // give up; the error is recorded below
        late = true;
        atomicOr(c.err, ERR_TIMEOUT);
      }
    }
    if (late) s_abort = 1;
  }
  __syncthreads();
  if (s_abort == 1) return;
  const uint32_t bpos = s_ts.bpos;
  const bool hasB = bpos < tn;
  const bool a_cont = s_ts.start[0] < tb;  // segment A began in an earlier tile
  const uint32_t wbase = (uint32_t)warp * 32 * ITEMS;

  // 2. rank within the warp among equal (segment, digit), in input order
  uint32_t key[ITEMS];
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t rnk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    const bool ok = p < tn;
    key[i] = ok ? s_keys[p] : 0u;
    const uint32_t bin =
        ok ? (((p >= bpos) ? (uint32_t)kRadix : 0u) | digit_of(key[i], c.shift)) : (uint32_t)BINS;
    uint32_t peers;  // ballots in plain passes, as in onesweep_pass
    if constexpr (Epi::kBallotRank) peers = warp_peers(bin, ok, kRadixBits + 1);
    else peers = __match_any_sync(0xffffffffu, bin);
    uint32_t before = 0;
    if (ok) before = s_whist[bin * WARPS + warp];
    __syncwarp();
    rnk[i] = before + __popc(peers & lt);
    if (ok && (peers & lt) == 0) s_whist[bin * WARPS + warp] = (uint16_t)(before + __popc(peers));
    __syncwarp();
  }
  __syncthreads();

  // 3. tile counts per bin; publish them for the tile's last segment at once
  uint32_t cA = 0, cB = 0;
  if (tid < kRadix) {
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t ta = s_whist[tid * WARPS + w], tb2 = s_whist[(kRadix + tid) * WARPS + w];
      s_whist[tid * WARPS + w] = (uint16_t)cA;
      s_whist[(kRadix + tid) * WARPS + w] = (uint16_t)cB;
      cA += ta;
      cB += tb2;
    }
    uint64_t* mine = c.status + (uint64_t)tile * kRadix + tid;
    if (hasB || !a_cont) st_relaxed_u64(mine, lb_pack(kFlagPre, c.epoch, hasB ? cB : cA));
    else st_relaxed_u64(mine, lb_pack(kFlagAgg, c.epoch, cA));
  }
  // 4. tile offsets of the bins (A bins, then B bins) and the segments' digit
  //    starts, two 64-bit scans
  uint32_t hA = 0, hB = 0;
  if (tid < kRadix) {
    hA = seg_hist[(uint64_t)s_ts.gid[0] * kRadix + tid];
    hB = hasB ? seg_hist[(uint64_t)s_ts.gid[1] * kRadix + tid] : 0u;
  }
  const uint64_t tsc = block_excl_scan64<THREADS>((uint64_t)cA | ((uint64_t)cB << 32), s_scan64);
  const uint64_t hsc = block_excl_scan64<THREADS>((uint64_t)hA | ((uint64_t)hB << 32), s_scan64);
  if (tid == kRadix - 1) s_totA = (uint32_t)tsc + cA;
  __syncthreads();
  uint32_t toffA = 0, toffB = 0;
  if (tid < kRadix) {
    toffA = (uint32_t)tsc;
    toffB = (uint32_t)(tsc >> 32) + s_totA;
    s_toff[tid] = toffA;
    s_toff[kRadix + tid] = toffB;
  }
  uint32_t val[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    val[i] = p < tn ? s_vals[p] : 0u;
  }
  __syncthreads();  // the input tile is consumed: its buffers take the output
  // 5. stage keys and values in bin order (tile-local positions need no
  //    global prefix)
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    if (p < tn) {
      const uint32_t bin = ((p >= bpos) ? (uint32_t)kRadix : 0u) | digit_of(key[i], c.shift);
      const uint32_t pos = s_toff[bin] + s_whist[bin * WARPS + warp] + rnk[i];
      s_keys[pos] = key[i];
      s_vals[pos] = val[i];
    }
  }
  // 6. look-back for segment A's digit prefixes
  if (tid < kRadix) {
    uint32_t prefA = 0;
    if (a_cont && s_abort == 0) {
      if (!look_back<16>(c, tile, tid, &prefA)) {
        atomicOr(c.err, ERR_TIMEOUT);
        s_abort = 1;
      }
      if (!hasB) st_relaxed_u64(c.status + (uint64_t)tile * kRadix + tid,
                                lb_pack(kFlagPre, c.epoch, prefA + cA));
    }
    s_gbase[tid] = s_ts.start[0] + (uint32_t)hsc + prefA - toffA;
    s_gbase[kRadix + tid] = s_ts.start[1] + (uint32_t)(hsc >> 32) - toffB;
  }
  __syncthreads();
  if (s_abort) return;

  // 7. write out: consecutive threads on consecutive slots of each bin's run
  const uint32_t totA = s_totA;
  for (uint32_t p = tid; p < tn; p += THREADS) {
    const uint32_t k = s_keys[p];
    const uint32_t seg = p >= totA ? 1u : 0u;
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
  static constexpr bool kBallotRank = true;
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
// Last pass of a per-dimension rank sort over one set: the sorted position of
// an item is its rank in that dimension.
struct SegEpiRank {
  static constexpr bool kNeedsUpdateInfo = false;
  static constexpr bool kBallotRank = false;
  RankOut out;
  __device__ void operator()(uint32_t, uint32_t v, uint32_t dest, uint32_t, const TileSegs&) const {
    out.put(v, dest, dest);
  }
};

struct SegEpiUpdate {
  static constexpr bool kNeedsUpdateInfo = true;
  static constexpr bool kBallotRank = false;
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
