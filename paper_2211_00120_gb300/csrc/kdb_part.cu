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
//   partition  every list is re-sorted by (new tag, key, index).  The new tag
//              is 2s+1 / 2s+2 by comparing the entry with the pivot (the tag
//              update of Sec. 3.2); since the list is already sorted by
//              (s, key, index), this is one stable radix pass on the child
//              bit within every segment.  The pass stages a tile in shared
//              memory by bulk copy, ranks left/right items with warp ballots,
//              finds the counts of earlier tiles of the same segment by
//              decoupled look-back (a warp reads 32 predecessors per round
//              trip), and writes both children's runs in order.
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
  const int d = a.mode == 0 ? x.l % a.k : a.dims[si.off + node];
  const uint32_t pos = e.base + y.seg_start(s_rel) + y.left_size(s_rel);
  if (d >= a.k || pos >= a.items) {
    atomicOr(x.err, ERR_INTERNAL);
    return;
  }
  const uint4 ent = a.lists[d][pos];
  a.piv[gid] = make_uint2(comp(ent, d), ent.w);
  a.perm[si.off + node] = ent.w;
}

// ---------------------------------------------------------------------------
constexpr int PT = kPartThreads;
constexpr int PI = kPartItems;
constexpr int PTILE = PT * PI;
constexpr int PW = PT / 32;

struct PartSeg {
  uint32_t start;   // first position of the segment in this level's array
  uint32_t ai, srel;
  uint32_t pk, po;  // pivot (key, original index)
  int dsplit;       // split dimension
  uint32_t csL, csR;  // first output position of the left / right child
  int mode;         // 0: next level's list, 1: original indices for the local finish
};

__device__ inline void part_seg_info(const PartArgs& a, uint32_t ai, uint32_t srel, uint32_t start,
                                     PartSeg* ps) {
  const LevelCtx& x = a.x;
  const ActiveEntry e = x.act[ai];
  const SetInfo si = x.sets[e.set];
  const LevelLayout y = LevelLayout::make(make_tree(si.n), x.l);
  ps->start = start;
  ps->ai = ai;
  ps->srel = srel;
  const uint2 pv = a.piv[(ai << x.l) | srel];
  ps->pk = pv.x;
  ps->po = pv.y;
  ps->dsplit = a.mode == 0 ? x.l % a.k : a.dims[si.off + full_nodes(x.l) + srel];
  uint32_t child0;
  if (e.next >= 0) {
    ps->mode = 0;
    child0 = x.act_next[e.next].base;
  } else {
    // the set continues in the local finish, which takes every list in
    // order as original indices
    ps->mode = 1;
    child0 = si.off;
  }
  ps->csL = child0 + (start - e.base) - srel;
  ps->csR = ps->csL + y.left_size(srel);
}

// Warp-parallel look-back: the lanes read the words of the 32 preceding
// tiles; values of consecutive published words are added until the nearest
// inclusive prefix.  Returns false if a wait ran past c.wait_ns.
__device__ inline bool warp_look_back(const PartArgs& a, uint32_t tile, uint32_t* prefix) {
  const int lane = threadIdx.x & 31;
  int64_t t = (int64_t)tile - 1;  // newest predecessor not yet consumed
  uint32_t acc = 0;
  bool waiting = false;
  uint64_t t0 = 0;
  for (;;) {
    const int64_t mine = t - lane;
    uint64_t w = mine >= 0 ? ld_relaxed_u64(a.status + mine) : lb_pack(kFlagPre, a.wait_epoch, 0);
    const uint32_t ep = (uint32_t)(w >> 32) & 0x3FFFFFFFu;
    const bool ready = ep == a.wait_epoch && (w >> 62) != 0;
    const bool pre = ready && (w >> 62) == 2;
    const uint32_t notready = __ballot_sync(0xffffffffu, !ready);
    const uint32_t pres = __ballot_sync(0xffffffffu, pre);
    const int first_nr = notready ? __ffs(notready) - 1 : 32;
    const int first_pre = pres ? __ffs(pres) - 1 : 32;
    if (first_pre < first_nr) {  // everything up to the prefix is published
      const uint32_t v = lane <= first_pre ? (uint32_t)w : 0u;
      *prefix = acc + __reduce_add_sync(0xffffffffu, v);
      return true;
    }
    if (first_nr > 0) {  // consume the published aggregates and move on
      const uint32_t v = lane < first_nr ? (uint32_t)w : 0u;
      acc += __reduce_add_sync(0xffffffffu, v);
      t -= first_nr;
      waiting = false;
      continue;
    }
    const uint64_t now = global_timer_ns();
    if (!waiting) {
      waiting = true;
      t0 = now;
    } else if (now - t0 > a.wait_ns) {
      *prefix = acc;
      return false;
    }
  }
}

__global__ void __launch_bounds__(PT, 6) partition_kernel(PartArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint4* s_in = reinterpret_cast<uint4*>(smem_raw);
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile, s_abort, s_bpos, s_acont;
  __shared__ PartSeg s_seg[2];
  __shared__ uint32_t s_wcnt[PW][6];  // per warp: LA RA LB RB PA PB
  __shared__ uint32_t s_woff[PW][4];
  __shared__ uint32_t s_prefL, s_prefP;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const LevelCtx& x = a.x;
  if (tid == 0) {
    s_abort = *reinterpret_cast<volatile uint32_t*>(x.err) != 0u;
    if (!s_abort) {
      const uint32_t tile = atomicAdd(a.ticket, 1u);
      s_tile = tile;
      const uint32_t tb = tile * (uint32_t)PTILE;
      const uint32_t tn = a.n - tb < (uint32_t)PTILE ? a.n - tb : (uint32_t)PTILE;
      mbar_init(&s_bar, 1);
      mbar_expect_tx(&s_bar, tn * 16u);
      bulk_g2s(s_in, a.in + tb, tn * 16u, &s_bar);
      uint32_t ai, sr, st, en;
      segment_at(x, tb, &ai, &sr, &st, &en);
      part_seg_info(a, ai, sr, st, &s_seg[0]);
      s_acont = st < tb;
      s_bpos = tn;
      if (en < tb + tn) {
        uint32_t a2, s2, st2, en2;
        segment_at(x, en, &a2, &s2, &st2, &en2);
        part_seg_info(a, a2, s2, st2, &s_seg[1]);
        s_bpos = en - tb;
        if (en2 < tb + tn) s_abort = 2;  // a segment shorter than a tile: not allowed
      } else {
        s_seg[1] = s_seg[0];
      }
    }
  }
  __syncthreads();
  if (s_abort == 1) return;
  if (s_abort == 2 && tid == 0) atomicOr(x.err, ERR_INTERNAL);
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
  const uint32_t bpos = s_bpos;
  const bool hasB = bpos < tn;
  const PartSeg sA = s_seg[0], sB = s_seg[1];

  // classify every item and rank it among its warp's items of the same
  // (segment, side), in list order
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t code[PI];  // bit 31: valid, bits 29-30: side (0 L, 1 R, 2 pivot), bit 28: B, low: rank
  uint32_t cnt[6] = {0, 0, 0, 0, 0, 0};
  const uint32_t wbase = (uint32_t)warp * 32 * PI;
#pragma unroll
  for (int i = 0; i < PI; ++i) {
    const uint32_t p = wbase + i * 32 + lane;
    const bool ok = p < tn;
    const bool isB = p >= bpos;
    uint32_t side = 3;
    if (ok) {
      const PartSeg& sg = isB ? sB : sA;
      const uint4 en = s_in[p];
      const uint32_t key = comp(en, sg.dsplit);
      side = before(key, en.w, sg.pk, sg.po) ? 0u : ((key == sg.pk && en.w == sg.po) ? 2u : 1u);
    }
    const uint32_t bLA = __ballot_sync(0xffffffffu, ok && !isB && side == 0);
    const uint32_t bRA = __ballot_sync(0xffffffffu, ok && !isB && side == 1);
    const uint32_t bLB = __ballot_sync(0xffffffffu, ok && isB && side == 0);
    const uint32_t bRB = __ballot_sync(0xffffffffu, ok && isB && side == 1);
    const uint32_t bPA = __ballot_sync(0xffffffffu, ok && !isB && side == 2);
    const uint32_t bPB = __ballot_sync(0xffffffffu, ok && isB && side == 2);
    uint32_t rank = 0;
    if (side == 0) rank = (isB ? cnt[2] + __popc(bLB & lt) : cnt[0] + __popc(bLA & lt));
    if (side == 1) rank = (isB ? cnt[3] + __popc(bRB & lt) : cnt[1] + __popc(bRA & lt));
    code[i] = (ok ? 0x80000000u : 0u) | (side << 29) | (isB ? 0x10000000u : 0u) | rank;
    cnt[0] += __popc(bLA);
    cnt[1] += __popc(bRA);
    cnt[2] += __popc(bLB);
    cnt[3] += __popc(bRB);
    cnt[4] += __popc(bPA);
    cnt[5] += __popc(bPB);
  }
  if (lane == 0)
    for (int q = 0; q < 6; ++q) s_wcnt[warp][q] = cnt[q];
  __syncthreads();
  if (tid == 0) {
    uint32_t run[4] = {0, 0, 0, 0}, pa = 0, pb = 0;
    for (int w = 0; w < PW; ++w) {
      for (int q = 0; q < 4; ++q) {
        s_woff[w][q] = run[q];
        run[q] += s_wcnt[w][q];
      }
      pa += s_wcnt[w][4];
      pb += s_wcnt[w][5];
    }
    // publish this tile's counts for its last segment: 2 * lefts + pivots
    uint64_t* mine = a.status + tile;
    if (hasB) st_relaxed_u64(mine, lb_pack(kFlagPre, a.epoch, 2 * run[2] + pb));
    else if (!s_acont) st_relaxed_u64(mine, lb_pack(kFlagPre, a.epoch, 2 * run[0] + pa));
    else st_relaxed_u64(mine, lb_pack(kFlagAgg, a.epoch, 2 * run[0] + pa));
    s_prefL = run[0];  // tile totals, replaced by the prefix below
    s_prefP = pa;
  }
  __syncthreads();
  if (warp == 0) {
    uint32_t v = 0;
    bool ok = true;
    if (s_acont) ok = warp_look_back(a, tile, &v);
    if (lane == 0) {
      if (!ok) {
        atomicOr(x.err, ERR_TIMEOUT);
        s_abort = 1;
      }
      if (s_acont && !hasB)
        st_relaxed_u64(a.status + tile, lb_pack(kFlagPre, a.epoch, v + 2 * s_prefL + s_prefP));
      s_prefL = v >> 1;
      s_prefP = v & 1u;
    }
  }
  __syncthreads();
  if (s_abort) return;

  // write every child's run in order
  const uint32_t prefL = s_prefL, prefR = (tb - sA.start) - s_prefL - s_prefP;
#pragma unroll
  for (int i = 0; i < PI; ++i) {
    const uint32_t cd = code[i];
    const uint32_t side = (cd >> 29) & 3u;
    if (!(cd & 0x80000000u) || side > 1) continue;
    const bool isB = (cd >> 28) & 1u;
    const PartSeg& sg = isB ? sB : sA;
    const uint32_t rank = cd & 0x0FFFFFFFu;
    uint32_t pos;
    if (side == 0) pos = sg.csL + (isB ? 0u : prefL) + s_woff[warp][isB ? 2 : 0] + rank;
    else pos = sg.csR + (isB ? 0u : prefR) + s_woff[warp][isB ? 3 : 1] + rank;
    const uint32_t lim = sg.mode == 0 ? a.next_items : a.total;
    if (pos >= lim) {
      atomicOr(x.err, ERR_INTERNAL);
      continue;
    }
    if (sg.mode == 0) a.out_next[pos] = s_in[wbase + i * 32 + lane];
    else a.out_lorig[(size_t)a.dlist * a.total + pos] = s_in[wbase + i * 32 + lane].w;
  }
}
}  // namespace

size_t partition_smem() { return (size_t)PTILE * 16; }

cudaError_t launch_pivots(const PivotArgs& a, cudaStream_t st) {
  const uint32_t nseg = a.x.nact << a.x.l;
  if (nseg == 0) return cudaSuccess;
  pivot_kernel<<<(nseg + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_partition(const PartArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const size_t smem = partition_smem();
  cudaError_t e =
      cudaFuncSetAttribute(partition_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (a.n + PTILE - 1) / PTILE;
  partition_kernel<<<tiles, PT, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace kdb
