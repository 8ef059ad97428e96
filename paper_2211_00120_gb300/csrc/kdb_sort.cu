// kdb_sort.cu -- instantiations of the onesweep pass and the fused tag update.
#include "kdb_launch.h"
#include "kdb_onesweep.cuh"
#include "kdb_segsort.cuh"

namespace kdb {

// Tag update of Sec. 3.2 applied while the level's last radix pass scatters.
// The sort key is (active set, subtree s_rel, rank in the split dimension), so
// `dest` is the item's position in the level-l sorted array and its subtree
// is read from the key.  With q = dest - sb(s) (Sec. 4.2) and the pivot rank
// p = ss(lChild(s)) (Observation 1):
//   q == p  -> the item is node s: pinned, written to its final slot;
//   q <  p  -> lChild(s);  q > p -> rChild(s).
// Children are written straight into the next level's compacted array
// (pinned items removed: one per earlier subtree of the level, plus this
// subtree's own pivot for right children), so the next level's tag is implied
// by position and never stored.  On a set's last sorted level the children
// are lowest-level nodes and go to their final slots.
struct EpiUpdate {
  static constexpr bool kBallotRank = false;
  LevelCtx x;
  uint32_t* perm;
  uint32_t* vals_next;
  __device__ void operator()(uint64_t key, uint32_t orig, uint32_t dest) const {
    const uint32_t ai = (uint32_t)(key >> (x.l + x.rb));
    const uint32_t s_rel = (uint32_t)(key >> x.rb) & ((1u << x.l) - 1u);
    if (ai >= x.nact) {
      atomicOr(x.err, ERR_INTERNAL);
      return;
    }
    const ActiveEntry e = x.act[ai];
    const SetInfo si = x.sets[e.set];
    const Tree t = make_tree(si.n);
    const LevelLayout y = LevelLayout::make(t, x.l);
    const uint32_t j = dest - e.base;
    const uint32_t q = j - y.seg_start(s_rel);
    const uint32_t pr = y.left_size(s_rel);
    // the item must lie inside its subtree's segment of its set
    if (j >= y.items || q >= y.seg_start(s_rel + 1) - y.seg_start(s_rel)) {
      atomicOr(x.err, ERR_INTERNAL);
      return;
    }
    if (q == pr) {
      perm[si.off + full_nodes(x.l) + s_rel] = orig;
      return;
    }
    const uint32_t jn = j - s_rel - (q > pr ? 1u : 0u);
    if (e.next < 0)
      perm[si.off + full_nodes(x.l + 1) + jn] = orig;
    else
      vals_next[x.act_next[e.next].base + jn] = orig;
  }
};

template <typename K, class Epi>
static cudaError_t run_pass(const K* kin, const uint32_t* vin, const Epi& epi, const PassCtl& c,
                            cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  auto kern = onesweep_pass<K, kSortThreads, kSortItems, Epi>;
  const size_t smem = OnesweepShape<K, kSortThreads, kSortItems>::kDynSmem;
  // the attribute belongs to the current device; set once per device
  cudaError_t e = ensure_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (c.n + kSortTile - 1) / kSortTile;
  kern<<<tiles, kSortThreads, smem, st>>>(kin, vin, c, epi);
  return cudaGetLastError();
}

cudaError_t pass_u64_pingpong(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                              uint32_t* vout, const PassCtl& c, cudaStream_t st) {
  return run_pass(kin, vin, EpiPingPong<uint64_t>{kout, vout}, c, st);
}
cudaError_t pass_u64_rank(const uint64_t* kin, const uint32_t* vin, const RankOut& out,
                          const SetInfo* sets, int set_shift, const PassCtl& c, cudaStream_t st) {
  return run_pass(kin, vin, EpiRank<uint64_t>{out, sets, set_shift}, c, st);
}
cudaError_t pass_u64_update(const uint64_t* kin, const uint32_t* vin, const LevelCtx& x,
                            uint32_t* perm, uint32_t* vals_next, const PassCtl& c,
                            cudaStream_t st) {
  return run_pass(kin, vin, EpiUpdate{x, perm, vals_next}, c, st);
}

template <class Epi>
static cudaError_t run_seg_pass(const uint32_t* kin, const uint32_t* vin, const LevelCtx& x,
                                const uint32_t* seg_hist, const Epi& epi, const PassCtl& c,
                                cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  auto kern = seg_onesweep_pass<kSegThreads, kSegItems, kSegMinBlocks, Epi>;
  const size_t smem = seg_pass_smem();
  cudaError_t e = ensure_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (c.n + kSegTile - 1) / kSegTile;
  kern<<<tiles, kSegThreads, smem, st>>>(kin, vin, c, x, seg_hist, epi);
  return cudaGetLastError();
}

cudaError_t seg_pass_pingpong(const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                              uint32_t* vout, const LevelCtx& x, const uint32_t* seg_hist,
                              const PassCtl& c, cudaStream_t st) {
  return run_seg_pass(kin, vin, x, seg_hist, SegEpiPingPong{kout, vout}, c, st);
}

size_t seg_pass_smem() {
  return (size_t)kSegTile * 8 + (size_t)2 * kRadix * (kSegThreads / 32) * 2;
}

cudaError_t seg_pass_rank(const uint32_t* kin, const uint32_t* vin, const LevelCtx& x,
                          const uint32_t* seg_hist, const RankOut& out, const PassCtl& c,
                          cudaStream_t st) {
  return run_seg_pass(kin, vin, x, seg_hist, SegEpiRank{out}, c, st);
}

cudaError_t seg_pass_update(const uint32_t* kin, const uint32_t* vin, const LevelCtx& x,
                            const uint32_t* seg_hist, uint32_t* perm, uint32_t* vals_next,
                            const PassCtl& c, cudaStream_t st) {
  return run_seg_pass(kin, vin, x, seg_hist, SegEpiUpdate{perm, vals_next, x.vals_local}, c, st);
}

}  // namespace kdb
