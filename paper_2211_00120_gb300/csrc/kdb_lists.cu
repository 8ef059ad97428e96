// kdb_lists.cu -- the level-0 sorted lists of the k <= 3 path.
//
// Every point is carried as a 16-byte entry: the order-preserving keys of its
// coordinates in dimensions 0..2 and its original index.  Comparing entries by
// (key_d, original index) is the paper's less() in dimension d (Sec. 3.1)
// with the tie rule.
//
// For every dimension d, list d is a stable LSD radix sort of the entries by
// key_d (4 passes of 8-bit digits, or 6 passes of 6-bit digits, each a
// segmented onesweep pass over 16-byte records, one segment per set) starting
// from input order, which leaves list d sorted by (key_d, original index): the
// order the level-0 sort produces when d is the root's split dimension.  For
// one set in round robin, the list of the level-1 dimension takes the side
// of the root's pivot into its last pass (rec_tag_pass) and so leaves sorted
// for level 1.
#include "kdb_launch.h"
#include "kdb_segsort.cuh"

namespace kdb {
namespace {

__device__ inline uint32_t comp(const uint4& e, int d) {
  return d == 0 ? e.x : (d == 1 ? e.y : e.z);
}
// ---------------------------------------------------------------------------
// Level-0 array of several sets: the entries of the sets that run global
// levels, back to back (a single set uses the input entries directly).
__global__ void gather_level0_kernel(ListBuildArgs a) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.items) return;
  if (*reinterpret_cast<volatile uint32_t*>(a.x.err)) return;
  const uint32_t ai = a.x.nact > 1 ? find_active_entry(a.x.act, a.x.nact, j) : 0;
  const ActiveEntry e = a.x.act[ai];
  const uint32_t src = a.x.sets[e.set].off + (j - e.base);
  if (src >= a.total) {
    atomicOr(a.x.err, ERR_INTERNAL);
    return;
  }
  a.out[j] = a.ents[src];
}

// Digit histograms of every (dimension, pass, segment) of the level-0 array;
// one block per chunk of one segment (a set).  BITS: the digit width.
template <int BITS>
__global__ void __launch_bounds__(256) rec_hist_kernel(RecHistArgs a) {
  constexpr int P = rec_passes(BITS);
  constexpr uint32_t R = 1u << BITS;
  __shared__ uint32_t s_hist[3 * P * R];
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
  const uint32_t n = x.sets[e.set].n;  // level 0: the whole set is one segment
  const uint32_t beg = e.base + (g - e.chunk0) * kSegChunk;
  const uint32_t end = min(e.base + n, beg + kSegChunk);
  if (beg >= end) return;
  const int H = a.k * P * (int)R;
  for (int i = threadIdx.x; i < H; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  for (uint32_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
    const uint4 en = a.ents[j];
    for (int d = 0; d < a.k; ++d) {
      const uint32_t key = comp(en, d);
#pragma unroll
      for (int p = 0; p < P; ++p) atomicAdd(&s_hist[(d * P + p) * R + ((key >> (BITS * p)) & (R - 1u))], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    const uint32_t v = s_hist[i];
    if (v) {
      const int dp = i / R, dg = i % R;  // dp = d * P + p
      atomicAdd(a.hist + ((uint64_t)dp * a.nseg + ai) * kRadixBins + dg, v);
    }
  }
}

// ---------------------------------------------------------------------------
// One stable LSD pass over 16-byte entries by digit (key_d >> shift) of BITS
// bits, every set its own segment.  The tile's records are staged by bulk copy; only
// their slot order is staged for the write-out, which reads the records from
// shared memory in digit order and writes each digit's run contiguously.
// The tile shape (threads RT, entries per thread RI, resident blocks RB) is a
// template parameter; the shapes built are listed in kRecShape.
// CNT: also count every entry's (side of the root's pivot, digit at
// cn.tshift) for the tagged last pass of the list (one set).
template <int RT, int RI, int RB, int BITS, bool CNT>
__global__ void __launch_bounds__(RT, RB)
    rec_sort_pass(const uint4* __restrict__ in, uint4* __restrict__ out, PassCtl c, LevelCtx x,
                  const uint32_t* __restrict__ seg_hist, int d, RecCount cn) {
  constexpr int RADIX = 1 << BITS;
  constexpr uint32_t DMASK = RADIX - 1;
  constexpr int BINS = 2 * RADIX;  // (segment A or B) x digit
  constexpr int RTILE = RT * RI;
  constexpr int RW = RT / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint4* s_rec = reinterpret_cast<uint4*>(smem_raw);
  uint16_t* s_slot = reinterpret_cast<uint16_t*>(s_rec + RTILE);
  uint16_t* s_whist = s_slot + RTILE;  // [RW][BINS]: a warp's digits on distinct banks
  __shared__ uint32_t s_gbase[BINS];
  __shared__ uint32_t s_toff[BINS];
  __shared__ uint64_t s_scan64[RW];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile, s_abort, s_totA;
  __shared__ TileSegs s_ts;
  __shared__ uint32_t s_thist[CNT ? 512 : 1];
  __shared__ uint2 s_piv;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if constexpr (CNT) {
    for (int i = tid; i < 512; i += RT) s_thist[i] = 0;
    if (tid == 0) s_piv = *cn.piv;
  }
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
      const uint32_t tb = tile * (uint32_t)RTILE;
      const uint32_t tn = c.n - tb < (uint32_t)RTILE ? c.n - tb : (uint32_t)RTILE;
      mbar_init(&s_bar, 1);
      mbar_expect_tx(&s_bar, tn * 16u);
      bulk_g2s(s_rec, in + tb, tn * 16u, &s_bar);
      uint32_t a, sr, st, en;
      segment_at(x, tb, &a, &sr, &st, &en);
      s_ts.ai[0] = a;
      s_ts.srel[0] = sr;
      s_ts.start[0] = st;
      s_ts.gid[0] = a;  // level 0: one segment per set
      s_ts.bpos = tn;
      if (en < tb + tn) {
        uint32_t a2, s2, st2, en2;
        segment_at(x, en, &a2, &s2, &st2, &en2);
        s_ts.ai[1] = a2;
        s_ts.srel[1] = s2;
        s_ts.start[1] = st2;
        s_ts.gid[1] = a2;
        s_ts.bpos = en - tb;
        if (en2 < tb + tn) s_abort = 2;
      } else {
        s_ts.ai[1] = a;
        s_ts.srel[1] = sr;
        s_ts.start[1] = st;
        s_ts.gid[1] = a;
      }
    }
  }
  for (int i = tid; i < BINS * RW / 2; i += RT) reinterpret_cast<uint32_t*>(s_whist)[i] = 0;
  __syncthreads();
  if (s_abort == 1) return;
  if (s_abort == 2 && tid == 0) atomicOr(c.err, ERR_INTERNAL);
  const uint32_t tile = s_tile;
  const uint32_t tb = tile * (uint32_t)RTILE;
  const uint32_t tn = c.n - tb < (uint32_t)RTILE ? c.n - tb : (uint32_t)RTILE;
  {
    bool waiting = false, late = false;
    uint64_t t0 = 0;
    while (!mbar_try_wait(&s_bar, 0)) {
      const uint64_t now = global_timer_ns();
      if (!waiting) {
        waiting = true;
        t0 = now;
      } else if (now - t0 > (late ? 2 : 1) * kCopyWaitNs) {
        if (late) break;
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
  const bool a_cont = s_ts.start[0] < tb;
  const uint32_t wbase = (uint32_t)warp * 32 * RI;
  const uint32_t lt = (1u << lane) - 1u;

  uint16_t bins[RI];
  uint16_t rnk[RI];
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    const bool ok = p < tn;
    uint32_t bin = BINS;
    if (ok) bin = ((p >= bpos) ? (uint32_t)RADIX : 0u) | ((comp(s_rec[p], d) >> c.shift) & DMASK);
    const uint32_t peers = warp_peers(bin, ok, BITS + 1);  // (segment, digit)
    uint32_t before = 0;
    if (ok) before = s_whist[warp * BINS + bin];
    __syncwarp();
    rnk[i] = (uint16_t)(before + __popc(peers & lt));
    if (ok && (peers & lt) == 0) s_whist[warp * BINS + bin] = (uint16_t)(before + __popc(peers));
    bins[i] = (uint16_t)bin;
    __syncwarp();
  }
  __syncthreads();
  uint32_t cA = 0, cB = 0;
  if (tid < RADIX) {
#pragma unroll
    for (int w = 0; w < RW; ++w) {
      const uint32_t ta = s_whist[w * BINS + tid], tb2 = s_whist[w * BINS + RADIX + tid];
      s_whist[w * BINS + tid] = (uint16_t)cA;
      s_whist[w * BINS + RADIX + tid] = (uint16_t)cB;
      cA += ta;
      cB += tb2;
    }
    uint64_t* mine = c.status + (uint64_t)tile * kRadix + tid;
    if (hasB || !a_cont) st_relaxed_u64(mine, lb_pack(kFlagPre, c.epoch, hasB ? cB : cA));
    else st_relaxed_u64(mine, lb_pack(kFlagAgg, c.epoch, cA));
  }
  uint32_t hA = 0, hB = 0;
  if (tid < RADIX) {
    hA = seg_hist[(uint64_t)s_ts.gid[0] * kRadix + tid];
    hB = hasB ? seg_hist[(uint64_t)s_ts.gid[1] * kRadix + tid] : 0u;
  }
  const uint64_t tsc = block_excl_scan64<RT>((uint64_t)cA | ((uint64_t)cB << 32), s_scan64);
  const uint64_t hsc = block_excl_scan64<RT>((uint64_t)hA | ((uint64_t)hB << 32), s_scan64);
  if (tid == RADIX - 1) s_totA = (uint32_t)tsc + cA;
  __syncthreads();
  uint32_t toffA = 0, toffB = 0;
  if (tid < RADIX) {
    toffA = (uint32_t)tsc;
    toffB = (uint32_t)(tsc >> 32) + s_totA;
    s_toff[tid] = toffA;
    s_toff[RADIX + tid] = toffB;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    if (p < tn) {
      const uint32_t bin = bins[i];
      s_slot[s_toff[bin] + s_whist[warp * BINS + bin] + rnk[i]] = (uint16_t)p;
    }
  }
  if (tid < RADIX) {
    uint32_t prefA = 0;
    if (a_cont && s_abort == 0) {
      if (!look_back<8>(c, tile, tid, &prefA)) {
        atomicOr(c.err, ERR_TIMEOUT);
        s_abort = 1;
      }
      if (!hasB) st_relaxed_u64(c.status + (uint64_t)tile * kRadix + tid,
                                lb_pack(kFlagPre, c.epoch, prefA + cA));
    }
    s_gbase[tid] = s_ts.start[0] + (uint32_t)hsc + prefA - toffA;
    s_gbase[RADIX + tid] = s_ts.start[1] + (uint32_t)(hsc >> 32) - toffB;
  }
  __syncthreads();
  if (s_abort) return;
  const uint32_t totA = s_totA;
  for (uint32_t sl = tid; sl < tn; sl += RT) {
    const uint4 rec = s_rec[s_slot[sl]];
    const uint32_t bin = (sl >= totA ? (uint32_t)RADIX : 0u) | ((comp(rec, d) >> c.shift) & DMASK);
    const uint32_t dest = s_gbase[bin] + sl;
    if (dest >= c.n) {
      atomicOr(c.err, ERR_INTERNAL);
      continue;
    }
    out[dest] = rec;
    if constexpr (CNT) {
      const uint32_t kp = comp(rec, cn.pdim);
      if (kp != s_piv.x || rec.w != s_piv.y) {  // the root is not counted
        const uint32_t side = (kp < s_piv.x || (kp == s_piv.x && rec.w < s_piv.y)) ? 0u : 1u;
        atomicAdd(&s_thist[(side << 8) | ((comp(rec, d) >> cn.tshift) & 255u)], 1u);
      }
    }
  }
  if constexpr (CNT) {
    __syncthreads();
    for (int i = tid; i < 512; i += RT)
      if (s_thist[i]) atomicAdd(&cn.thist[i], s_thist[i]);
  }
}

// ---------------------------------------------------------------------------
// The last digit pass of list D1 of one set, sorted by (side of the root's
// pivot, digit) instead of the digit alone.  The passes before it left the
// list sorted by (lower digits, index), so this stable pass leaves it sorted
// by (side, key, index): the order of level 1's sort in dimension D1, the
// left subtree's points first (Sec. 3.1 with the tag update of Sec. 3.2
// applied once) -- the list arrives on level 1 without a partition pass.
// The root itself (the pivot) is dropped.  Each side's digit counts have
// their own look-back words (c: side 0, c1: side 1) and global bases from
// thist, counted by the list's first pass.
template <int RT, int RI, int RB>
__global__ void __launch_bounds__(RT, RB)
    rec_tag_pass(const uint4* __restrict__ in, uint4* __restrict__ out, PassCtl c, PassCtl c1,
                 const uint2* __restrict__ piv, int pdim, const uint32_t* __restrict__ thist, int d) {
  static_assert(RT == kRadix, "one thread per digit of each side");
  constexpr int RADIX = 256;
  constexpr int BINS = 2 * RADIX;  // (side, digit)
  constexpr int RTILE = RT * RI;
  constexpr int RW = RT / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint4* s_rec = reinterpret_cast<uint4*>(smem_raw);
  uint16_t* s_slot = reinterpret_cast<uint16_t*>(s_rec + RTILE);
  uint16_t* s_whist = s_slot + RTILE;  // [RW][BINS]
  __shared__ uint32_t s_gbase[BINS];
  __shared__ uint32_t s_toff[BINS];
  __shared__ uint64_t s_scan64[RW];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile, s_abort, s_tot0, s_tot, s_left;
  __shared__ uint2 s_piv;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_abort = *reinterpret_cast<volatile uint32_t*>(c.err) != 0u;
    if (!s_abort) {
      s_tile = atomicAdd(c.ticket, 1u);
      if ((uint64_t)(s_tile + 1) * kRadix > c.status_words || (uint64_t)(s_tile + 1) * kRadix > c1.status_words) {
        atomicOr(c.err, ERR_INTERNAL);  // the last tiles: no tile waits on them
        s_abort = 1;
      }
    }
    if (!s_abort) {
      const uint32_t tb = s_tile * (uint32_t)RTILE;
      const uint32_t tn = c.n - tb < (uint32_t)RTILE ? c.n - tb : (uint32_t)RTILE;
      mbar_init(&s_bar, 1);
      mbar_expect_tx(&s_bar, tn * 16u);
      bulk_g2s(s_rec, in + tb, tn * 16u, &s_bar);
      s_piv = *piv;
    }
  }
  for (int i = tid; i < BINS * RW / 2; i += RT) reinterpret_cast<uint32_t*>(s_whist)[i] = 0;
  __syncthreads();
  if (s_abort) return;
  const uint32_t tile = s_tile;
  const uint32_t tb = tile * (uint32_t)RTILE;
  const uint32_t tn = c.n - tb < (uint32_t)RTILE ? c.n - tb : (uint32_t)RTILE;
  {
    bool waiting = false, late = false;
    uint64_t t0 = 0;
    while (!mbar_try_wait(&s_bar, 0)) {
      const uint64_t now = global_timer_ns();
      if (!waiting) {
        waiting = true;
        t0 = now;
      } else if (now - t0 > (late ? 2 : 1) * kCopyWaitNs) {
        if (late) break;
        late = true;
        atomicOr(c.err, ERR_TIMEOUT);
      }
    }
    if (late) s_abort = 1;
  }
  __syncthreads();
  if (s_abort) return;
  const uint2 pv = s_piv;
  const uint32_t wbase = (uint32_t)warp * 32 * RI;
  const uint32_t lt = (1u << lane) - 1u;

  uint16_t bins[RI];
  uint16_t rnk[RI];
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    uint32_t bin = BINS;  // out of range, or the root
    if (p < tn) {
      const uint4 e = s_rec[p];
      const uint32_t kp = comp(e, pdim);
      if (kp != pv.x || e.w != pv.y) {
        const uint32_t side = (kp < pv.x || (kp == pv.x && e.w < pv.y)) ? 0u : 1u;  // 0: left of the root
        bin = (side << 8) | ((comp(e, d) >> c.shift) & 255u);
      }
    }
    const bool ok = bin < BINS;
    const uint32_t peers = warp_peers(bin, ok, 9);  // (side, digit)
    uint32_t before = 0;
    if (ok) before = s_whist[warp * BINS + bin];
    __syncwarp();
    rnk[i] = (uint16_t)(before + __popc(peers & lt));
    if (ok && (peers & lt) == 0) s_whist[warp * BINS + bin] = (uint16_t)(before + __popc(peers));
    bins[i] = (uint16_t)bin;
    __syncwarp();
  }
  __syncthreads();
  // thread t: digit t of side 0 (bin t) and of side 1 (bin 256 + t)
  uint32_t cA = 0, cB = 0;
#pragma unroll
  for (int w = 0; w < RW; ++w) {
    const uint32_t ta = s_whist[w * BINS + tid], tb2 = s_whist[w * BINS + RADIX + tid];
    s_whist[w * BINS + tid] = (uint16_t)cA;
    s_whist[w * BINS + RADIX + tid] = (uint16_t)cB;
    cA += ta;
    cB += tb2;
  }
  {
    const uint64_t f = tile == 0 ? kFlagPre : kFlagAgg;
    st_relaxed_u64(c.status + (uint64_t)tile * kRadix + tid, lb_pack(f, c.epoch, cA));
    st_relaxed_u64(c1.status + (uint64_t)tile * kRadix + tid, lb_pack(f, c1.epoch, cB));
  }
  const uint32_t hA = thist[tid], hB = thist[RADIX + tid];
  const uint64_t tsc = block_excl_scan64<RT>((uint64_t)cA | ((uint64_t)cB << 32), s_scan64);
  const uint64_t hsc = block_excl_scan64<RT>((uint64_t)hA | ((uint64_t)hB << 32), s_scan64);
  if (tid == RADIX - 1) {
    s_tot0 = (uint32_t)tsc + cA;
    s_tot = s_tot0 + (uint32_t)(tsc >> 32) + cB;
    s_left = (uint32_t)hsc + hA;  // points on the left of the root: its left subtree's size
  }
  __syncthreads();
  const uint32_t toffA = (uint32_t)tsc, toffB = (uint32_t)(tsc >> 32) + s_tot0;
  s_toff[tid] = toffA;
  s_toff[RADIX + tid] = toffB;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    const uint32_t bin = bins[i];
    if (p < tn && bin < BINS) s_slot[s_toff[bin] + s_whist[warp * BINS + bin] + rnk[i]] = (uint16_t)p;
  }
  uint32_t prefA = 0, prefB = 0;
  if (tile > 0) {
    const bool okA = look_back<8>(c, tile, tid, &prefA);
    const bool okB = look_back<8>(c1, tile, tid, &prefB);
    if (!okA || !okB) {
      atomicOr(c.err, ERR_TIMEOUT);
      s_abort = 1;
    }
    st_relaxed_u64(c.status + (uint64_t)tile * kRadix + tid, lb_pack(kFlagPre, c.epoch, prefA + cA));
    st_relaxed_u64(c1.status + (uint64_t)tile * kRadix + tid, lb_pack(kFlagPre, c1.epoch, prefB + cB));
  }
  s_gbase[tid] = (uint32_t)hsc + prefA - toffA;
  s_gbase[RADIX + tid] = s_left + (uint32_t)(hsc >> 32) + prefB - toffB;
  __syncthreads();
  if (s_abort) return;
  const uint32_t tot0 = s_tot0, tot = s_tot, nout = c.n - 1;
  for (uint32_t sl = tid; sl < tot; sl += RT) {
    const uint4 rec = s_rec[s_slot[sl]];
    const uint32_t bin = (sl >= tot0 ? (uint32_t)RADIX : 0u) | ((comp(rec, d) >> c.shift) & 255u);
    const uint32_t dest = s_gbase[bin] + sl;
    if (dest >= nout) {
      atomicOr(c.err, ERR_INTERNAL);
      continue;
    }
    out[dest] = rec;
  }
}

}  // namespace

size_t rec_sort_smem(int shape) {
  const TileShape& sh = kRecShape[shape];
  return (size_t)sh.threads * sh.items * 18 + (size_t)2 * kRadix * (sh.threads / 32) * 2;
}
uint32_t rec_sort_tile() { return (uint32_t)kRecTileMin; }

cudaError_t launch_gather_level0(const ListBuildArgs& a, cudaStream_t st) {
  if (a.items == 0) return cudaSuccess;
  gather_level0_kernel<<<(a.items + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rec_hist(const RecHistArgs& a, cudaStream_t st) {
  if (a.chunks == 0) return cudaSuccess;
  static_assert(kRecDigitWidths == 2, "one launcher per width");
  if (a.bits == 6) rec_hist_kernel<6><<<a.chunks, 256, 0, st>>>(a);
  else rec_hist_kernel<8><<<a.chunks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <int S, int BITS, bool CNT>
cudaError_t launch_rec_sort_shape(const uint4* in, uint4* out, const PassCtl& c, const LevelCtx& x,
                                  const uint32_t* seg_hist, int d, const RecCount& cn, cudaStream_t st) {
  constexpr TileShape sh = kRecShape[S];
  const size_t smem = rec_sort_smem(S);
  const void* fn = (const void*)rec_sort_pass<sh.threads, sh.items, sh.blocks, BITS, CNT>;
  cudaError_t e = ensure_smem(fn, smem);
  if (e != cudaSuccess) return e;
  const uint32_t tile = (uint32_t)(sh.threads * sh.items);
  const uint32_t tiles = (c.n + tile - 1) / tile;
  rec_sort_pass<sh.threads, sh.items, sh.blocks, BITS, CNT><<<tiles, sh.threads, smem, st>>>(in, out, c, x,
                                                                                              seg_hist, d, cn);
  return cudaGetLastError();
}

cudaError_t launch_rec_sort_pass(const uint4* in, uint4* out, const PassCtl& c, const LevelCtx& x,
                                 const uint32_t* seg_hist, int d, int shape, int bits, cudaStream_t st,
                                 const RecCount* count) {
  if (c.n == 0) return cudaSuccess;
  static_assert(kRecShapes == 2 && kRecDigitWidths == 2, "one launcher per shape and width");
  const RecCount cn = count ? *count : RecCount{};
  if (count && count->thist) {  // the counting first pass of list D1: 8-bit digits only
    if (bits != 8) return cudaErrorInvalidValue;
    if (shape == 1) return launch_rec_sort_shape<1, 8, true>(in, out, c, x, seg_hist, d, cn, st);
    return launch_rec_sort_shape<0, 8, true>(in, out, c, x, seg_hist, d, cn, st);
  }
  if (bits == 6) {
    if (shape == 1) return launch_rec_sort_shape<1, 6, false>(in, out, c, x, seg_hist, d, cn, st);
    return launch_rec_sort_shape<0, 6, false>(in, out, c, x, seg_hist, d, cn, st);
  }
  if (shape == 1) return launch_rec_sort_shape<1, 8, false>(in, out, c, x, seg_hist, d, cn, st);
  return launch_rec_sort_shape<0, 8, false>(in, out, c, x, seg_hist, d, cn, st);
}

cudaError_t launch_rec_tag_pass(const uint4* in, uint4* out, const PassCtl& c, const PassCtl& c1, const uint2* piv,
                                int pdim, const uint32_t* thist, int d, int shape, cudaStream_t st) {
  (void)shape;  // one thread per digit of each side: the 256-thread shape
  if (c.n == 0) return cudaSuccess;
  constexpr TileShape sh = kRecShape[0];
  static_assert(sh.threads == kRadix && sh.threads * sh.items == kRecTileMin, "the smallest tile, 256 threads");
  const size_t smem = rec_sort_smem(0);
  const void* fn = (const void*)rec_tag_pass<sh.threads, sh.items, sh.blocks>;
  cudaError_t e = ensure_smem(fn, smem);
  if (e != cudaSuccess) return e;
  const uint32_t tile = (uint32_t)(sh.threads * sh.items);
  const uint32_t tiles = (c.n + tile - 1) / tile;
  rec_tag_pass<sh.threads, sh.items, sh.blocks><<<tiles, sh.threads, smem, st>>>(in, out, c, c1, piv, pdim, thist, d);
  return cudaGetLastError();
}

}  // namespace kdb
