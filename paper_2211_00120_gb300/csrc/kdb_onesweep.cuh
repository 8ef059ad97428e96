// kdb_onesweep.cuh -- one pass of a stable LSD "onesweep" radix sort.
//
// The paper's per-level step is a whole-array sort by (tag, coordinate)
// (Sec. 3.1); Sec. 7.1 suggests replacing its comparator sort by a radix sort
// over a packed integer key.  This is that sort's pass kernel: an 8-bit digit,
// one tile of TILE items per thread block, tiles handed out in launch order by
// an atomic ticket so that every tile a block waits on has already started.
//
// Per tile:
//   1. load keys (and values) coalesced, warp-striped;
//   2. rank each key among equal digits inside its warp (per-bit ballots, or
//      __match_any_sync where the epilogue is heavy: warp-level multi-split), per-warp digit counters in shared memory;
//   3. tile-wide digit counts and offsets by a block scan;
//   4. publish the tile's digit counts, stage the tile in shared memory in
//      digit order, then decoupled look-back: add up the counts of earlier
//      tiles (16 per round trip) until one with an inclusive prefix is found,
//      publish the inclusive prefix.  Each wait is bounded by a time limit; on
//      expiry the tile records ERR_TIMEOUT, publishes a prefix so that later
//      tiles do not wait on it, and writes nothing;
//   5. write the tile out with consecutive threads on consecutive positions
//      of each digit's run.
// The epilogue object decides what is written for each (key, value, dest).
#pragma once

#include "kdb_internal.cuh"

namespace kdb {

constexpr int kRadixBits = 8;
constexpr int kRadix = kRadixBins;
static_assert((1 << kRadixBits) == kRadixBins, "digit width");

struct PassCtl {
  uint32_t n;             // items
  int shift;              // bit offset of this pass's digit
  const uint32_t* hist;   // kRadix counts of this digit over all n items
  uint64_t* status;       // per tile, per digit look-back words
  uint32_t* ticket;       // tile ticket, 0 on entry
  uint32_t epoch;         // unique per pass in a build, 1 .. 2^30-1
  uint32_t wait_epoch;    // epoch waited for (== epoch unless a fault is injected)
  uint64_t wait_ns;       // bound on one look-back wait
  uint32_t* err;          // device status word
  uint64_t status_words;  // capacity of status: a tile whose words lie beyond it does nothing
};

// look-back word: [63:62] flag, [61:32] epoch, [31:0] count
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPre = 2ull << 62;
__device__ inline uint64_t lb_pack(uint64_t flag, uint32_t epoch, uint32_t v) {
  return flag | ((uint64_t)(epoch & 0x3FFFFFFFu) << 32) | v;
}

template <typename K>
__device__ inline uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & (kRadix - 1);
}

// Exclusive scan of one value per thread over the whole block (values of
// threads that do not take part are passed as 0).  Returns the exclusive
// prefix; *total receives the block sum.
template <int THREADS>
__device__ inline uint32_t block_excl_scan(uint32_t v, uint32_t* s_tmp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < THREADS / 32 ? s_tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < THREADS / 32) s_tmp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const uint32_t before = warp ? s_tmp[warp - 1] : 0;
  *total = s_tmp[THREADS / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// Look back from tile-1 for digit `tid`: adds predecessors' counts until one
// carries an inclusive prefix.  WIN predecessor words are read per round trip,
// so the inclusive-prefix frontier moves WIN tiles per L2 round trip instead
// of one.  Returns false if a wait ran past c.wait_ns.
template <int WIN>
__device__ inline bool look_back(const PassCtl& c, uint32_t tile, int tid, uint32_t* prefix) {
  int64_t t = (int64_t)tile - 1;
  uint32_t acc = 0;
  bool waiting = false;
  uint64_t t0 = 0;
  for (;;) {
    uint64_t w[WIN];
#pragma unroll
    for (int i = 0; i < WIN; ++i)
      w[i] = (t - i >= 0) ? ld_relaxed_u64(c.status + (uint64_t)(t - i) * kRadix + tid)
                          : lb_pack(kFlagPre, c.wait_epoch, 0);
    int used = 0;
    bool done = false;
#pragma unroll
    for (int i = 0; i < WIN; ++i) {
      if (done || used < i) break;
      const uint64_t x = w[i];
      const uint32_t ep = (uint32_t)(x >> 32) & 0x3FFFFFFFu;
      if (ep != c.wait_epoch || (x >> 62) == 0) break;  // not published yet
      acc += (uint32_t)x;
      ++used;
      if ((x >> 62) == 2 || t - i == 0) done = true;
    }
    if (done) {
      *prefix = acc;
      return true;
    }
    if (used > 0) {
      t -= used;
      waiting = false;
      continue;
    }
    const uint64_t now = global_timer_ns();
    if (!waiting) {
      waiting = true;
      t0 = now;
    } else if (now - t0 > c.wait_ns) {
      *prefix = acc;
      return false;
    }
  }
}

template <typename K, int THREADS, int ITEMS>
struct OnesweepShape {
  static constexpr int kTile = THREADS * ITEMS;
  static constexpr size_t kDynSmem = (size_t)kTile * (sizeof(K) + sizeof(uint32_t));
};

template <typename K, int THREADS, int ITEMS, class Epi>
__global__ void __launch_bounds__(THREADS)
    onesweep_pass(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, PassCtl c,
                  Epi epi) {
  static_assert(THREADS >= kRadix && THREADS % 32 == 0, "one thread per digit");
  constexpr int WARPS = THREADS / 32;
  constexpr int TILE = THREADS * ITEMS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + TILE);
  __shared__ uint32_t s_whist[WARPS][kRadix];
  __shared__ uint32_t s_toff[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_scan[WARPS];
  __shared__ uint32_t s_tile, s_abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    // after any device error the inputs may be garbage: do nothing.  A block
    // that leaves here has taken no ticket, so no tile ever waits on it.
    s_abort = *reinterpret_cast<volatile uint32_t*>(c.err) != 0u;
    if (!s_abort) {
      s_tile = atomicAdd(c.ticket, 1u);
      // the last tiles: no tile waits on them
      if ((uint64_t)(s_tile + 1) * kRadix > c.status_words) {
        atomicOr(c.err, ERR_INTERNAL);
        s_abort = 1;
      }
    }
  }
  for (int i = tid; i < WARPS * kRadix; i += THREADS) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  if (s_abort) return;
  const uint32_t tile = s_tile;
  const uint64_t tbase = (uint64_t)tile * TILE;
  const uint32_t tn = (uint32_t)((uint64_t)c.n - tbase < (uint64_t)TILE ? (uint64_t)c.n - tbase : TILE);
  const uint32_t wbase = (uint32_t)warp * 32 * ITEMS;

  K key[ITEMS];
  uint32_t val[ITEMS];
  uint32_t rnk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    if (p < tn) {
      key[i] = keys_in[tbase + p];
      val[i] = vals_in ? vals_in[tbase + p] : (uint32_t)(tbase + p);
    }
  }

  // 2. warp-level multi-split ranking, in input order (stable)
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    const bool ok = p < tn;
    const uint32_t d = ok ? digit_of(key[i], c.shift) : (uint32_t)kRadix;
    // plain passes: eight ballots (up to 256 digits in a warp, where
    // match.any is slow); passes with a heavier epilogue: match.any, which
    // needs fewer registers
    uint32_t peers;
    if constexpr (Epi::kBallotRank) peers = warp_peers(d, ok, kRadixBits);
    else peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (ok) before = s_whist[warp][d];
    __syncwarp();
    if (ok) {
      rnk[i] = before + __popc(peers & lt);
      if ((peers & lt) == 0) s_whist[warp][d] = before + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();

  // 3. per digit: warp-exclusive offsets, tile count, tile offsets
  uint32_t cnt = 0;
  if (tid < kRadix) {
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t t = s_whist[w][tid];
      s_whist[w][tid] = cnt;
      cnt += t;
    }
  }
  uint32_t dummy;
  const uint32_t toff = block_excl_scan<THREADS>(tid < kRadix ? cnt : 0u, s_scan, &dummy);
  const uint32_t bstart =
      block_excl_scan<THREADS>(tid < kRadix ? c.hist[tid] : 0u, s_scan, &dummy);

  // 4. publish this tile's counts, stage the tile in digit order (tile-local
  //    positions need no global prefix), then look back
  if (tid < kRadix) {
    s_toff[tid] = toff;
    st_relaxed_u64(c.status + (uint64_t)tile * kRadix + tid,
                   lb_pack(tile == 0 ? kFlagPre : kFlagAgg, c.epoch, cnt));
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    if (p < tn) {
      const uint32_t d = digit_of(key[i], c.shift);
      const uint32_t pos = s_toff[d] + s_whist[warp][d] + rnk[i];
      s_keys[pos] = key[i];
      s_vals[pos] = val[i];
    }
  }
  if (tid < kRadix) {
    uint32_t prefix = 0;
    if (tile > 0) {
      if (!look_back<16>(c, tile, tid, &prefix)) {
        atomicOr(c.err, ERR_TIMEOUT);
        s_abort = 1;
      }
      st_relaxed_u64(c.status + (uint64_t)tile * kRadix + tid,
                     lb_pack(kFlagPre, c.epoch, prefix + cnt));
    }
    s_gbase[tid] = bstart + prefix - toff;  // modulo 2^32: dest = s_gbase[d] + p
  }
  __syncthreads();
  if (s_abort) return;

  // 5. write out: consecutive threads on consecutive slots of each digit's run
  for (uint32_t p = tid; p < tn; p += THREADS) {
    const K k = s_keys[p];
    const uint32_t d = digit_of(k, c.shift);
    const uint32_t dest = s_gbase[d] + p;
    if (dest >= c.n) {
      atomicOr(c.err, ERR_INTERNAL);
      continue;
    }
    epi(k, s_vals[p], dest);
  }
}

// ---- epilogues ------------------------------------------------------------
template <typename K>
struct EpiPingPong {
  static constexpr bool kBallotRank = true;
  K* keys_out;
  uint32_t* vals_out;
  __device__ void operator()(K k, uint32_t v, uint32_t dest) const {
    keys_out[dest] = k;
    vals_out[dest] = v;
  }
};

// Last pass of the per-dimension coordinate sort: the sorted position of an
// item, less its set's first sorted position, is its rank in that dimension.
template <typename K>
struct EpiRank {
  static constexpr bool kBallotRank = false;
  RankOut out;
  const SetInfo* sets;     // nullptr for a single set starting at 0
  int set_shift;           // set id = key >> set_shift (multi-set keys)
  __device__ void operator()(K k, uint32_t v, uint32_t dest) const {
    uint32_t base = 0;
    if (sets) base = sets[(uint32_t)((uint64_t)k >> set_shift)].off;
    out.put(v, dest - base, dest);
  }
};

}  // namespace kdb
