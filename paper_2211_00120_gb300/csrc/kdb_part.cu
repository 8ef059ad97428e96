// kdb_part.cu -- the per-level child-bit pass of the k <= 3 path.
//
// Every point is carried as a 16-byte entry: the order-preserving keys of its
// coordinates in dimensions 0..2 and its original index.  Comparing entries by
// (key_d, original index) is the paper's less() in dimension d (Sec. 3.1)
// with the tie rule, so no rank table is needed.  Level 0 starts from the
// per-dimension sorted lists (kdb_lists.cu).
//
// Level l: list d holds the live points sorted by (subtree tag, key_d, index),
// the order the paper's level-l sort produces when d is the split dimension
// (Sec. 3.1, Observation 3).
//   pivot      for every subtree s the entry at rank ss(lChild(s)) of s's
//              segment in the list of s's split dimension is node s
//              (Observation 1): pinned;
//   partition  a list is advanced b = 1 .. 3 levels at once: re-sorted by
//              (tag b levels down, key, index).  Each step of the tag update
//              (Sec. 3.2) sends an entry to 2s+1 / 2s+2 by comparing it with
//              the pivot of s; since the list is already sorted by
//              (s, key, index), the b steps together are one stable split of
//              every segment into its 2^b descendants' runs.  The pass stages
//              a tile in shared memory by bulk copy (its shape a template
//              argument), ranks the entries per (segment, descendant) with
//              warp match_any, finds the counts of earlier tiles of the same
//              segment by decoupled look-back (lane groups read several
//              predecessors per round trip), and writes every descendant's
//              run in order.
#include "kdb_launch.h"
#include "kdb_segsort.cuh"

namespace kdb {
namespace {

__device__ inline uint32_t comp(const uint4& e, int d) {
  return d == 0 ? e.x : (d == 1 ? e.y : e.z);
}
// (key, index) of entry e in dimension d strictly below the pivot (pk, po)?
__device__ inline bool before(uint32_t key, uint32_t idx, uint32_t pk, uint32_t po) {
  return key < pk || (key == pk && idx < po);
}

// ---------------------------------------------------------------------------
// Pivot of every subtree of level l (Observation 1): pinned at node s.
__global__ void pivot_kernel(PivotArgs a) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  const LevelCtx& x = a.x;
  if (gid >= (x.nact << x.l)) return;
  if (*reinterpret_cast<volatile uint32_t*>(x.err)) return;
  const uint32_t ai = gid >> x.l, s_rel = gid & ((1u << x.l) - 1u);
  const ActiveEntry e = x.act[ai];
  const SetInfo si = x.sets[e.set];
  const LevelLayout y = LevelLayout::make(make_tree(si.n), x.l);
  const uint32_t node = full_nodes(x.l) + s_rel;
  const int d = a.mode == 0 ? (x.l + x.dim0) % a.k : a.dims[si.off + node];
  const uint32_t pos = e.base + y.seg_start(s_rel) + y.left_size(s_rel);
  if (d >= a.k || pos >= a.items) {
    atomicOr(x.err, ERR_INTERNAL);
    return;
  }
  const uint4 ent = a.lists[d][pos];
  a.piv[gid] = make_uint2(comp(ent, d), ent.w);
  a.perm[si.off + node] = ent.w;
  if (a.pts_out) write_record_from_entry(a.pts_out + (uint64_t)(si.off + node) * a.stride, ent, a.k, a.ctype);
}

// ---------------------------------------------------------------------------
// Tight-box rule: split dimension of subtree c of level l + 1 = the widest
// side of the box of its points.  List d of level l + 1 is sorted by
// (subtree, key_d, index), so the subtree's smallest and largest key_d are
// its first and last entries: the per-subtree min/max reduction costs two
// reads per dimension.  Extent arithmetic as for the clipped domain: float32
// hi - lo (exact differences for integer coordinates), strict '>' from d = 0.
__global__ void tight_children_kernel(TightArgs a) {
  const LevelCtx& x = a.x;
  const int lc = x.l + 1;
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (x.nact << lc)) return;
  if (*reinterpret_cast<volatile uint32_t*>(x.err)) return;
  const uint32_t ei = gid >> lc, c_rel = gid & ((1u << lc) - 1u);
  const ActiveEntry e = x.act[ei];
  if (e.next < 0) return;  // the set's next level runs in the local finish
  const SetInfo si = x.sets[e.set];
  const Tree tree = make_tree(si.n);
  const uint32_t node = full_nodes(lc) + c_rel;
  if (node >= si.n) return;
  const LevelLayout y = LevelLayout::make(tree, lc);
  const uint32_t base = x.act_next[e.next].base;
  const uint32_t first = base + y.seg_start(c_rel), end = base + y.seg_start(c_rel + 1);
  if (end <= first || end > a.items_next) {
    atomicOr(x.err, ERR_INTERNAL);
    return;
  }
  uint32_t lo[3], hi[3];
  for (int d = 0; d < a.k; ++d) {
    lo[d] = comp(a.lists[d][first], d);
    hi[d] = comp(a.lists[d][end - 1], d);
  }
  a.dims[si.off + node] = (uint8_t)widest_of_keys(lo, hi, a.k, a.ctype);
}

// ---------------------------------------------------------------------------
constexpr int NB = 2 * kLiftBins;  // bins of a tile: (segment A or B) x child
static_assert(kLiftMax == 3, "pivot tables hold depth-3 subtrees");

struct LiftSeg {
  uint32_t start;              // first position of the segment in the level-p array
  uint32_t left0;              // ss(lChild) of the segment's root: its pivot's rank
  uint32_t cs[kLiftBins];      // first output position of each child's run
  uint32_t pk[kLiftBins - 1];  // pivots of the segment's first bs levels, heap order
  uint32_t po[kLiftBins - 1];
  uint8_t dim[kLiftBins - 1];  // their split dimensions
  int bs;                      // levels the segment descends: b, or fewer where its set
                               // leaves the active list on the way
  int mode;                    // 0: next level's list, 1: original indices for the local finish
};

// The segment holding position j of level p, with its bounds (the set's
// tables from the arguments for a single set, else from the active list).
__device__ inline void part_segment_at(const PartArgs& a, uint32_t j, uint32_t* ai, uint32_t* srel,
                                       uint32_t* start, uint32_t* end) {
  if (!a.single) {
    segment_at(a.x, j, ai, srel, start, end);
    return;
  }
  const LevelLayout y = LevelLayout::make(make_tree(a.set0.n), a.x.l);
  const uint32_t s = y.seg_of(j - a.act0.base);
  *ai = 0;
  *srel = s;
  *start = a.act0.base + y.seg_start(s);
  *end = a.act0.base + y.seg_start(s + 1);
}

// One segment's setup, by the 16 lanes hl = 0..15 of a half warp: lanes
// 0..7 the first output position of each descendant's run, lanes 8..14 the
// pivots (and split dimensions) of the segment's first bs levels, lane 0 the
// rest; the pivot loads are issued side by side.  Every lane first follows
// the set through the active lists of levels p + 1 .. p + b - 1: the set
// descends while it is active (bs levels), and its pivots of level p + e sit
// at its index in that level's active list.
__device__ inline void lift_seg_info(const PartArgs& a, uint32_t ai, uint32_t srel, uint32_t start,
                                     LiftSeg* ps, uint32_t hl) {
  const LevelCtx& x = a.x;
  const ActiveEntry e = a.single ? a.act0 : x.act[ai];
  const SetInfo si = a.single ? a.set0 : x.sets[e.set];
  const Tree tree = make_tree(si.n);
  uint32_t idx[kLiftMax];
  idx[0] = ai;
  int bs = 1;
  int32_t nxt = e.next;  // the set's index on level p + bs, -1 if it is not active there
  while (bs < a.b && nxt >= 0) {
    idx[bs] = (uint32_t)nxt;
    nxt = a.act_mid[bs - 1][nxt].next;
    ++bs;
  }
  const int mode = (a.handoff || nxt < 0) ? 1 : 0;  // mode 0: bs = b, nxt its index on p + b
  const uint32_t nb = 1u << bs;
  if (hl == 0) {
    ps->start = start;
    ps->mode = mode;
    ps->bs = bs;
    ps->left0 = LevelLayout::make(tree, x.l).left_size(srel);
  }
  if (hl < nb) {
    uint32_t base_out;
    if (mode == 1) base_out = si.off;
    else base_out = a.single ? a.out_base0 : a.act_out[nxt].base;
    const LevelLayout yo = LevelLayout::make(tree, x.l + bs);
    ps->cs[hl] = base_out + yo.seg_start((srel << bs) + hl);
  }
  if (hl >= kLiftBins && hl - kLiftBins + 1 < nb) {
    const uint32_t h = hl - kLiftBins;
    const int e2 = 31 - __clz(h + 1);  // depth of heap node h below the segment
    const uint32_t rel = (srel << e2) + (h + 1 - (1u << e2));
    const int lq = x.l + e2;
    const uint2 pv = a.piv[e2][(idx[e2] << lq) | rel];
    ps->pk[h] = pv.x;
    ps->po[h] = pv.y;
    ps->dim[h] = (uint8_t)(a.mode == 0 ? (lq + x.dim0) % a.k : a.dims[si.off + full_nodes(lq) + rel]);
  }
}

// Warp-parallel decoupled look-back over nbin bins: lane group g (32 / nbin
// lanes) takes bin g, each lane reading R consecutive predecessor words, so
// a group covers R * 32 / nbin predecessors per round trip; it adds published
// values up to the nearest inclusive prefix.  Writes the exclusive prefix of
// every bin to s_pref; false if a wait ran past wait_ns.
template <int R>
__device__ inline bool warp_look_back_bins(const PartArgs& a, uint32_t tile, int nbin,
                                           uint32_t* s_pref) {
  const int lane = threadIdx.x & 31;
  const int lpb = 32 / nbin;
  const int g = lane / lpb, j = lane % lpb;
  const uint32_t gmask = lpb == 32 ? 0xffffffffu : (((1u << lpb) - 1u) << (g * lpb));
  int64_t t = (int64_t)tile - 1;  // newest predecessor not yet consumed (group-uniform)
  uint32_t acc = 0;
  bool done = false, ok = true, waiting = false;
  uint64_t t0 = 0;
  for (;;) {
    // this lane's words: positions j * R + r back from t
    uint64_t w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t mine = t - (int64_t)(j * R + r);
      w[r] = lb_pack(kFlagPre, a.wait_epoch, 0);
      if (!done && mine >= 0) w[r] = ld_relaxed_u64(a.status + (uint64_t)mine * kLiftBins + g);
    }
    int fnr = R, fpr = R;  // the lane's first word not ready, first inclusive prefix
    uint32_t v[R];
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      const uint32_t ep = (uint32_t)(w[r] >> 32) & 0x3FFFFFFFu;
      const bool ready = done || (ep == a.wait_epoch && (w[r] >> 62) != 0);
      const bool pre = !done && ready && (w[r] >> 62) == 2;
      v[r] = done ? 0u : (uint32_t)w[r];
      if (!ready) fnr = r;
      if (pre) fpr = r;
    }
    const uint32_t nr = __ballot_sync(0xffffffffu, fnr < R) & gmask;
    const uint32_t pr = __ballot_sync(0xffffffffu, fpr < R) & gmask;
    const int jn = nr ? __ffs(nr) - 1 - g * lpb : lpb;
    const int jp = pr ? __ffs(pr) - 1 - g * lpb : lpb;
    int FNR = jn * R, FPR = jp * R;  // the group's first word not ready, first prefix
    if (R > 1) {
      FNR += __shfl_sync(0xffffffffu, fnr, g * lpb + (jn < lpb ? jn : 0)) % R;
      FPR += __shfl_sync(0xffffffffu, fpr, g * lpb + (jp < lpb ? jp : 0)) % R;
    }
    uint32_t s1 = 0, s2 = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int pos = j * R + r;
      if (pos <= FPR) s1 += v[r];
      if (pos < FNR) s2 += v[r];
    }
    for (int o = 1; o < lpb; o <<= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (!done) {
      if (FPR < FNR) {  // everything up to the prefix is published
        acc += s1;
        done = true;
      } else if (FNR > 0) {  // consume the published aggregates and move on
        acc += s2;
        t -= FNR;
        waiting = false;
      } else {
        const uint64_t now = global_timer_ns();
        if (!waiting) {
          waiting = true;
          t0 = now;
        } else if (now - t0 > a.wait_ns) {
          ok = false;
          done = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
  if (j == 0) s_pref[g] = acc;
  return __all_sync(0xffffffffu, ok);
}

// One pass that advances list dlist by b levels (1 <= b <= 3): the tag update
// of Sec. 3.2 applied b times with the pivots of levels p .. p+b-1, and the
// list re-sorted by the new tag.  The list is sorted by (tag_p, key, index),
// so the new order is a stable split of every segment into its 2^b
// descendants' runs; items pinned on the way are dropped.
template <int PT, int PI, int PB>
__global__ void __launch_bounds__(PT, PB) partition_kernel(PartArgs a) {
  constexpr int PTILE = PT * PI;
  constexpr int PW = PT / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint4* s_in = reinterpret_cast<uint4*>(smem_raw);
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile, s_abort, s_bpos, s_acont;
  __shared__ LiftSeg s_seg[2];
  __shared__ uint32_t s_wcnt[PW][NB];  // per warp and bin: items, then exclusive offsets
  __shared__ uint32_t s_tcnt[NB];      // tile totals per bin
  __shared__ uint32_t s_prefA[kLiftBins];
  __shared__ uint32_t s_wbase[PW][NB];  // per warp and bin: first output position

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const LevelCtx& x = a.x;
  const int nbin = 1 << a.b;
  // tile setup by warp 0: lane 0 takes the ticket and issues the bulk copy,
  // then the two half warps fill in segments A and B side by side (B = A
  // when the tile lies in one segment)
  if (warp == 0) {
    uint32_t tile = 0, ab = 0;
    if (lane == 0) {
      ab = *reinterpret_cast<volatile uint32_t*>(x.err) != 0u;
      if (!ab) {
        tile = atomicAdd(a.ticket, 1u);
        if ((uint64_t)(tile + 1) * kLiftBins > a.status_words) {  // the last tiles: no tile waits on them
          atomicOr(x.err, ERR_INTERNAL);
          ab = 1;
        }
      }
    }
    tile = __shfl_sync(0xffffffffu, tile, 0);
    ab = __shfl_sync(0xffffffffu, ab, 0);
    if (!ab) {
      const uint32_t tb = tile * (uint32_t)PTILE;
      const uint32_t tn = a.n - tb < (uint32_t)PTILE ? a.n - tb : (uint32_t)PTILE;
      if (lane == 0) {
        mbar_init(&s_bar, 1);
        mbar_expect_tx(&s_bar, tn * 16u);
        bulk_g2s(s_in, a.in + tb, tn * 16u, &s_bar);
      }
      uint32_t ai, sr, st, en;
      part_segment_at(a, tb, &ai, &sr, &st, &en);
      const bool hasB = en < tb + tn;
      uint32_t a2 = ai, s2 = sr, st2 = st, en2 = en;
      if (hasB) part_segment_at(a, en, &a2, &s2, &st2, &en2);
      const uint32_t half = (uint32_t)lane >> 4;
      lift_seg_info(a, half ? a2 : ai, half ? s2 : sr, half ? st2 : st, &s_seg[half], (uint32_t)lane & 15u);
      if (lane == 0) {
        s_acont = st < tb;
        s_bpos = hasB ? en - tb : tn;
        if (hasB && en2 < tb + tn) ab = 2;  // a segment shorter than a tile: not allowed
      }
    }
    if (lane == 0) {
      s_tile = tile;
      s_abort = ab;
    }
  }
  for (int i = tid; i < PW * NB; i += PT) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();
  if (s_abort == 1) return;  // no copy was issued
  const uint32_t tile = s_tile;
  const uint32_t tb = tile * (uint32_t)PTILE;
  const uint32_t tn = a.n - tb < (uint32_t)PTILE ? a.n - tb : (uint32_t)PTILE;
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
        atomicOr(x.err, ERR_TIMEOUT);
      }
    }
    if (late) s_abort = 1;
  }
  __syncthreads();
  if (s_abort == 1) return;
  if (s_abort == 2) {  // the copy has landed; nothing else is in flight
    if (tid == 0) atomicOr(x.err, ERR_INTERNAL);
    return;
  }
  const uint32_t bpos = s_bpos;
  const bool hasB = bpos < tn;

  // classify every item (child path or pinned) and rank it among its warp's
  // items of the same (segment, child), in list order
  const uint32_t lt = (1u << lane) - 1u;
  uint16_t bins[PI];
  uint16_t rnk[PI];
  const uint32_t wbase = (uint32_t)warp * 32 * PI;
#pragma unroll
  for (int i = 0; i < PI; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    uint32_t bin = NB;  // not written: out of range or pinned
    if (p < tn) {
      const uint32_t sg = p >= bpos ? 1u : 0u;
      const LiftSeg& S = s_seg[sg];
      const uint4 en = s_in[p];
      uint32_t h = 0;
      bool pinned = false;
      int e2 = 0;
      if (a.pos_first) {
        // the list is in the split order of level p: the item's rank in its
        // segment decides its side (Observation 1), no comparison needed
        const uint32_t q = tb + p - S.start;
        pinned = q == S.left0;
        h = q < S.left0 ? 1u : 2u;
        e2 = 1;
      }
      for (; e2 < S.bs && !pinned; ++e2) {
        const uint32_t key = comp(en, S.dim[h]);
        const uint32_t pk = S.pk[h], po = S.po[h];
        if (key == pk && en.w == po) {
          pinned = true;
          break;
        }
        h = 2 * h + (before(key, en.w, pk, po) ? 1u : 2u);
      }
      if (!pinned) bin = sg * kLiftBins + (h - ((1u << S.bs) - 1u));
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, bin);
    uint32_t prev = 0;
    if (bin < NB) prev = s_wcnt[warp][bin];
    __syncwarp();
    rnk[i] = (uint16_t)(prev + __popc(peers & lt));
    if (bin < NB && (peers & lt) == 0) s_wcnt[warp][bin] = prev + __popc(peers);
    bins[i] = (uint16_t)bin;
    __syncwarp();
  }
  __syncthreads();
  if (tid < NB) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < PW; ++w) {
      const uint32_t c = s_wcnt[w][tid];
      s_wcnt[w][tid] = run;
      run += c;
    }
    s_tcnt[tid] = run;
  }
  __syncthreads();
  // publish the counts of this tile's last segment: B's (which starts here),
  // or A's -- an inclusive prefix if A starts here, else an aggregate
  const bool a_cont = s_acont != 0;
  if (tid < nbin) {
    uint64_t* mine = a.status + (uint64_t)tile * kLiftBins + tid;
    if (hasB) st_relaxed_u64(mine, lb_pack(kFlagPre, a.epoch, s_tcnt[kLiftBins + tid]));
    else st_relaxed_u64(mine, lb_pack(a_cont ? kFlagAgg : kFlagPre, a.epoch, s_tcnt[tid]));
  }
  if (warp == 0) {
    bool ok = true;
    // three-level lifts (four lanes per child): two words a lane, eight
    // predecessors a round trip; otherwise one word a lane
    if (a_cont) ok = nbin == kLiftBins ? warp_look_back_bins<2>(a, tile, nbin, s_prefA)
                                       : warp_look_back_bins<1>(a, tile, nbin, s_prefA);
    else if (lane < kLiftBins) s_prefA[lane] = 0;
    __syncwarp();
    if (lane < nbin) {
      if (a_cont && !hasB)
        st_relaxed_u64(a.status + (uint64_t)tile * kLiftBins + lane,
                       lb_pack(kFlagPre, a.epoch, s_prefA[lane] + s_tcnt[lane]));
    }
    if (!ok && lane == 0) {
      atomicOr(x.err, ERR_TIMEOUT);
      s_abort = 1;
    }
  }
  __syncthreads();
  if (s_abort) return;
  // where each warp's items of each bin start in the output: the child's
  // run, the earlier tiles' items of the child (segment A), the earlier warps'
  for (int i = tid; i < PW * NB; i += PT) {
    const int w = i / NB, bin = i % NB, sg = bin / kLiftBins, c = bin % kLiftBins;
    s_wbase[w][bin] = s_seg[sg].cs[c] + (sg ? 0u : s_prefA[c]) + s_wcnt[w][bin];
  }
  const int modeA = s_seg[0].mode, modeB = s_seg[1].mode;
  __syncthreads();

  // write every child's run in order
#pragma unroll
  for (int i = 0; i < PI; ++i) {
    const uint32_t bin = bins[i];
    if (bin >= NB) continue;
    const int mode = bin >= (uint32_t)kLiftBins ? modeB : modeA;
    const uint32_t pos = s_wbase[warp][bin] + rnk[i];
    const uint32_t lim = mode == 0 ? a.next_items : a.total;
    if (pos >= lim) {
      atomicOr(x.err, ERR_INTERNAL);
      continue;
    }
    const uint4 en = s_in[wbase + i * 32 + lane];
    if (mode == 0) a.out_next[pos] = en;
    else if (a.out_lents && a.dlist == 0) a.out_lents[pos] = en;
    else a.out_lorig[(size_t)a.dlist * a.total + pos] = en.w;
  }
}
}  // namespace

size_t partition_smem(int shape) {
  return (size_t)kPartShape[shape].threads * kPartShape[shape].items * 16;
}

cudaError_t launch_pivots(const PivotArgs& a, cudaStream_t st) {
  const uint32_t nseg = a.x.nact << a.x.l;
  if (nseg == 0) return cudaSuccess;
  pivot_kernel<<<(nseg + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tight_children(const TightArgs& a, cudaStream_t st) {
  const uint32_t n = a.x.nact << (a.x.l + 1);
  if (n == 0) return cudaSuccess;
  tight_children_kernel<<<(n + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_partition_shape(const PartArgs& a, cudaStream_t st) {
  constexpr TileShape sh = kPartShape[S];
  const size_t smem = partition_smem(S);
  cudaError_t e = ensure_smem((const void*)partition_kernel<sh.threads, sh.items, sh.blocks>, smem);
  if (e != cudaSuccess) return e;
  const uint32_t tile = (uint32_t)(sh.threads * sh.items);
  const uint32_t tiles = (a.n + tile - 1) / tile;
  partition_kernel<sh.threads, sh.items, sh.blocks><<<tiles, sh.threads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_partition(const PartArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  static_assert(kPartShapes == 3, "one launcher per shape");
  switch (a.shape) {
    case 1: return launch_partition_shape<1>(a, st);
    case 2: return launch_partition_shape<2>(a, st);
    default: return launch_partition_shape<0>(a, st);
  }
}

}  // namespace kdb
