// kdb_launch.h -- host-side launchers of the builder's kernels (internal).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "kdb_internal.cuh"

namespace kdb {

// Everything one level of the build needs to know about its sets.
struct LevelCtx {
  const SetInfo* sets;
  const ActiveEntry* act;       // active sets of level l (device)
  const ActiveEntry* act_next;  // active sets of level l+1 (device), may be empty
  uint32_t nact;
  int l;
  int dim0;        // round robin: level l splits in dimension (l + dim0) mod k
  int rb;          // bits of a rank
  uint32_t* err;   // device status word: kernels do nothing once it is set
  int local_next;  // 1: a set that leaves the active list goes to the local finish
  uint32_t* vals_local;  // per set at its first record: the local level's items
};

struct PassCtl;

// Raises a kernel's dynamic shared-memory limit on the current device if it
// is below `bytes`; remembers what it set, so that later launches (also
// inside a stream capture) make no attribute call.
cudaError_t ensure_smem(const void* func, size_t bytes);

// Presorted-list levels (kdb_part.cu), k <= 3: one 16-byte entry per point
// (order-preserving keys of coordinates 0..2, original index), one list per
// dimension.
// Tile shapes of the two sort kernels: threads x items per thread at a
// number of resident blocks per SM.  Each kernel is compiled for a few
// measured shapes; the autotuner (kdb_autotune) times them on a problem and
// keeps the fastest, shape 0 being the default.  Measured at 1e8 float3
// round robin (record sort ranking by ballots, partition tiles set up by
// warp 0): partition 256 x 13 at four blocks per SM 10.47 ms, 512 x 13 at two
// 10.74 ms; record sort 256 x 13 at three 10.30 ms, 512 x 8 at two 10.42 ms,
// 384 x 11 at two 10.52 ms, 256 x 16 at two 11.65 ms, 256 x 9 at four
// 12.87 ms.
struct TileShape {
  int threads, items, blocks;
};
constexpr int kPartShapes = 3;
constexpr TileShape kPartShape[kPartShapes] = {{256, 13, 4}, {512, 13, 2}, {128, 13, 8}};
constexpr int kRecShapes = 2;
constexpr TileShape kRecShape[kRecShapes] = {{256, 13, 3}, {512, 8, 2}};
// smallest tile of each kernel: the look-back buffers are sized for it.  A
// partition tile stays below 2^13 - 1 entries, so it holds at most two
// segments of a global level.
constexpr int kPartTile = 128 * 13;
constexpr int kRecTileMin = 256 * 13;
static_assert(kRecTileMin <= 512 * 8, "the smallest record-sort tile");
static_assert(512 * 13 < (1 << 13) - 1, "partition tiles hold at most two segments");
// Digit widths of the level-0 sort: a 32-bit key takes rec_passes(bits)
// passes.  Histograms and look-back words keep a stride of kRadixBins per
// (pass, segment) and per tile whatever the width.
constexpr int kRecDigitWidths = 2;
constexpr int kRecDigitBits[kRecDigitWidths] = {8, 6};
constexpr int kRecMaxPasses = 6;
constexpr int rec_passes(int bits) { return (32 + bits - 1) / bits; }
static_assert(rec_passes(8) <= kRecMaxPasses && rec_passes(6) <= kRecMaxPasses, "passes");
struct ListBuildArgs {      // level-0 array of several sets
  LevelCtx x;               // level 0
  uint32_t items;
  const uint4* ents;        // entries in input order
  uint4* out;
  uint32_t total;
};
struct RecHistArgs {        // digit histograms per (dimension, pass, set)
  LevelCtx x;               // level 0 (chunk0 / cps filled in)
  uint32_t chunks;
  const uint4* ents;        // level-0 array
  uint32_t* hist;           // [k * passes][nseg][256]
  uint32_t nseg;
  int k;
  int bits;                 // digit width: one of kRecDigitBits
};
struct PivotArgs {
  LevelCtx x;
  const uint4* lists[3];    // this level's lists
  uint32_t items;
  uint2* piv;               // out: pivot (key, original index) per segment
  uint32_t* perm;           // out: node -> original index
  const uint8_t* dims;      // widest: split dimension per node
  int k, mode;
  unsigned char* pts_out;   // records written directly at their nodes (stride = 4k), or nullptr
  int stride;
  int ctype;                // coordinate type (kCoordF32 / I32 / U32)
};
// Tight-box split rule: split dimension of every subtree of level l + 1 of
// the sets that stay on the global levels, from their first and last entries
// in each list of level l + 1 (kdb_part.cu).
struct TightArgs {
  LevelCtx x;               // level l (x.act, x.act_next)
  const uint4* lists[3];    // the lists of level l + 1
  uint32_t items_next;      // items of level l + 1
  uint8_t* dims;
  int k;
  int ctype;                // coordinate type: integers have exact extents
};
cudaError_t launch_tight_children(const TightArgs& a, cudaStream_t st);
// One partition pass advances a list by 1..kLiftMax levels at once.
constexpr int kLiftMax = 3;
constexpr int kLiftBins = 1 << kLiftMax;  // descendants of a segment kLiftMax levels down
struct PartArgs {
  LevelCtx x;               // level p, the input list's level
  const ActiveEntry* act_out;  // active sets of level p + b
  const ActiveEntry* act_mid[kLiftMax - 1];  // active sets of levels p + 1, p + 2 (or nullptr)
  int b;                    // levels to advance, 1..kLiftMax; a set that leaves the
                            // active list before p + b stops there (its local finish)
  int pos_first;            // 1: the list is in level p's split order (its dimension is
                            // level p's), so the first level goes by position
  int shape;                // tile shape: index into kPartShape
  int handoff;              // 1: every set goes to the local finish (at level p + b,
                            // or earlier where it leaves the active list)
  const uint4* in;          // list sorted by (tag on level p, key_dlist, index)
  uint4* out_next;          // the list on level p + b
  uint32_t* out_lorig;      // original indices for the local finish (sets leaving),
                            // one array of `total` per list
  uint4* out_lents;         // if set: list 0 is handed over as whole entries here
  const uint2* piv[kLiftMax];  // pivots (key, index) of levels p .. p + b - 1
  const uint8_t* dims;
  int k, mode, dlist;
  uint32_t n, next_items, total;
  uint64_t* status;         // kLiftBins look-back words per tile
  uint32_t* ticket;
  uint32_t epoch, wait_epoch;
  uint64_t wait_ns;
  uint64_t status_words;    // capacity of status
  // one set (single = 1): its tables, so that a tile's setup reads no memory
  int single;
  SetInfo set0;
  ActiveEntry act0;         // the set's entry on level p
  uint32_t out_base0;       // the set's first position in the list on level p + b
};
size_t partition_smem(int shape);
// The first pass of list D1 can also count, for the tagged last pass of that
// list (rec_tag_pass), every entry's (side of the root's pivot, last digit)
// into thist[512]; the root itself is not counted.
struct RecCount {
  const uint2* piv;   // the root's pivot (key in dimension pdim, index)
  int pdim;           // the root's split dimension
  uint32_t* thist;    // [2][256], added to; nullptr: no counting
  int tshift;         // bit offset of the last digit
};
size_t rec_sort_smem(int shape);
uint32_t rec_sort_tile();  // entries of the smallest record-sort tile (one look-back word per digit each)
cudaError_t launch_gather_level0(const ListBuildArgs& a, cudaStream_t st);
cudaError_t launch_rec_hist(const RecHistArgs& a, cudaStream_t st);
cudaError_t launch_rec_sort_pass(const uint4* in, uint4* out, const PassCtl& c, const LevelCtx& x,
                                 const uint32_t* seg_hist, int d, int shape, int bits, cudaStream_t st,
                                 const RecCount* count = nullptr);
// The last pass of list D1 of one set, sorted by (side of the root's pivot,
// digit): the list leaves the pass on level 1, the root dropped (n - 1
// entries out).  c1: the look-back words of the second side (c1.status a
// region of its own).
cudaError_t launch_rec_tag_pass(const uint4* in, uint4* out, const PassCtl& c, const PassCtl& c1, const uint2* piv,
                                int pdim, const uint32_t* thist, int d, int shape, cudaStream_t st);
cudaError_t launch_pivots(const PivotArgs& a, cudaStream_t st);
cudaError_t launch_partition(const PartArgs& a, cudaStream_t st);

// Local finish of small subtrees (kdb_local.cu).
constexpr int kLocalThreads = 1024;
#ifndef KDB_LOCAL_LOG
#define KDB_LOCAL_LOG 13
#endif
constexpr int kLocalLog = KDB_LOCAL_LOG;          // subtrees of <= 2^13 - 1 points
constexpr int kLocalCap = 1 << kLocalLog;         // 8192
constexpr int kLocalMax = kLocalCap - 1;
constexpr int kLocalMaxK = 4;                     // shared-memory budget: k + 1 lists
struct LocalSet {
  uint32_t off, n;
  int l0;          // level at which the set's subtrees are finished locally
  uint32_t lbox0;  // first slot of its subtrees' domains in the local box array
};
struct LocalWork {
  uint32_t set;
  uint32_t s_rel;  // subtree index on level l0 of that set
};
struct LocalArgs {
  const LocalWork* work;
  uint32_t nwork;
  const LocalSet* lsets;
  const uint32_t* vals_local;   // original indices (rank arrays gathered), or
  const uint32_t* lorig;        // k <= 3: per dimension the original indices of the
                                // items leaving the global levels, in list order
  const uint4* lents;           // if set: list 0 as whole entries (replaces lorig[0])
  const uint4* rows;            // entries in input order (sets local from level 0)
  const uint32_t* ranks;
  uint32_t total;
  int k, mode;
  const unsigned char* pts;
  int stride;
  const float* boxes_local;  // widest: domain of each local root with l0 > 0
  const uint32_t* bbox;      // widest: scene box keys per set (roots with l0 = 0)
  uint8_t* dims;
  uint32_t* perm;
  uint32_t* err;
  unsigned char* pts_out;    // records written directly at their nodes (stride = 4k), or nullptr
  int ctype;                 // coordinate type (kCoordF32 / I32 / U32)
  int dim0;                  // round robin: level l splits in dimension (l + dim0) mod k
};
size_t local_smem_bytes(int k);
cudaError_t launch_local_finish(const LocalArgs& a, cudaStream_t st);

// Radix pass geometry (one tile per block).
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
// Segmented passes: 256 threads x 15 items = 3840 < 2^13 - 1, the shortest
// subtree segment of a segmented level, so a tile touches at most two
// segments; three blocks per SM.
constexpr int kSegThreads = 256;
constexpr int kSegItems = 15;
constexpr int kSegMinBlocks = 3;
constexpr int kSegTile = kSegThreads * kSegItems;
size_t seg_pass_smem();


// onesweep passes (kdb_sort.cu)
cudaError_t pass_u64_pingpong(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                              uint32_t* vout, const PassCtl& c, cudaStream_t st);
cudaError_t pass_u64_rank(const uint64_t* kin, const uint32_t* vin, const RankOut& out,
                          const SetInfo* sets, int set_shift, const PassCtl& c, cudaStream_t st);
cudaError_t pass_u64_update(const uint64_t* kin, const uint32_t* vin, const LevelCtx& x,
                            uint32_t* perm, uint32_t* vals_next, const PassCtl& c,
                            cudaStream_t st);

// segmented passes over 32-bit rank keys (kdb_sort.cu); every segment of the
// level must be at least one tile long
cudaError_t seg_pass_pingpong(const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                              uint32_t* vout, const LevelCtx& x, const uint32_t* seg_hist,
                              const PassCtl& c, cudaStream_t st);
cudaError_t seg_pass_update(const uint32_t* kin, const uint32_t* vin, const LevelCtx& x,
                            const uint32_t* seg_hist, uint32_t* perm, uint32_t* vals_next,
                            const PassCtl& c, cudaStream_t st);
// last pass of a one-set rank sort (x describes one segment: the whole array)
cudaError_t seg_pass_rank(const uint32_t* kin, const uint32_t* vin, const LevelCtx& x,
                          const uint32_t* seg_hist, const RankOut& out, const PassCtl& c,
                          cudaStream_t st);

// Sharded single-tree build (kdb_dist.cu): the steps of the top levels on
// one shard of the points.
constexpr int kDistMaxDest = 64;  // nodes of a top level, destinations of the exchange
struct DistArgs {
  const unsigned char* pts;
  uint32_t n;               // points of the shard
  int k, stride, ctype;
  int32_t* tags;            // per point: node (heap index) on the current level, -1 once pinned
  uint32_t first, nodes;    // the level's first node and its node count (or first destination node, count)
  const uint8_t* node_dim;  // split dimension per node of the level
  const uint64_t* prefix;   // radix select: per node the key bits fixed so far
  int prefix_bits;
  uint32_t index_base;      // original index of the shard's first point
  uint32_t* hist;           // [nodes][256]
  uint32_t* box;            // [nodes][2k] coordinate keys: min, then max
  const uint64_t* pivot;    // per node its pivot's key (coordinate key << 32 | original index)
  int64_t* pinned;          // per node the shard position of its pivot (if on this shard)
  uint32_t* block_counts;   // [blocks][nodes]
  const uint32_t* block_offsets;  // [blocks][nodes]: first output position
  unsigned char* out_pts;
  uint32_t* out_index;
  uint32_t* err;
};
uint32_t dist_blocks(uint32_t n, int sms);
cudaError_t launch_dist_hist(const DistArgs& a, int sms, cudaStream_t st);
cudaError_t launch_dist_box(const DistArgs& a, int sms, cudaStream_t st);
cudaError_t launch_dist_assign(const DistArgs& a, int sms, cudaStream_t st);
cudaError_t launch_dist_count(const DistArgs& a, uint32_t blocks, cudaStream_t st);
cudaError_t launch_dist_scatter(const DistArgs& a, uint32_t blocks, cudaStream_t st);
// Memory-lean build: a subtree built in its own level order (in a slice of
// the partitioned records) written to its nodes of the whole tree.
struct LeanPlaceArgs {
  const unsigned char* src;  // the subtree's m records, its level order
  unsigned char* dst;        // the whole tree's records
  uint32_t m, total;         // subtree nodes, tree nodes
  int g;                     // the subtree's root is node F(g) + rank
  uint32_t rank;
  int stride;
  uint32_t* err;
};
cudaError_t launch_lean_place(const LeanPlaceArgs& a, cudaStream_t st);
// Memory-lean build: the original indices of every node's points whose
// coordinate key equals the node's (a.prefix, 32 bits), up to `cap` per node
// (out[node * cap + j]; counts[node] = all of them, zeroed by the caller).
cudaError_t launch_lean_collect(const DistArgs& a, uint32_t cap, uint32_t* counts, uint32_t* out, int sms,
                                cudaStream_t st);
// ERR_NAN in *err if a float coordinate of the n records is NaN.
cudaError_t launch_nan_check(const unsigned char* pts, uint32_t n, int k, int stride, uint32_t* err, int sms,
                             cudaStream_t st);

// tree kernels (kdb_tree.cu)
struct PrepassArgs {
  const unsigned char* pts;
  uint32_t total;       // records
  int k, stride;
  const SetInfo* sets;  // nsets entries
  uint32_t nsets;
  uint32_t* keys32;     // k * total (single set) or nullptr
  uint64_t* keys64;     // k * total (several sets) or nullptr
  uint64_t kstride;     // elements between two dimensions' keys (>= total)
  uint4* ents;          // k <= 3: entries (keys of dims 0..2, index) or nullptr
  uint32_t* hist;       // k * passes * 256, or nullptr
  int passes;
  uint32_t* bbox;       // nsets * 2k (min keys, then max keys) or nullptr
  uint32_t* err;
  int ctype;            // coordinate type (kCoordF32 / I32 / U32)
  uint32_t beg, end;    // records [beg, end) of this launch (end = 0: all of them)
  // one set of entries (prepass_fuses_rec_hist): the digit histograms of the
  // level-0 list sort ([k * passes][256], added to), or nullptr
  uint32_t* rec_hist;
  int rec_bits;         // their digit width
};
cudaError_t launch_prepass(const PrepassArgs& a, int num_sms, cudaStream_t st);
// Whether launch_prepass takes the vectorised kernel for these arguments,
// which also counts the level-0 digit histograms when rec_hist is given.
bool prepass_fuses_rec_hist(const PrepassArgs& a);

struct LevelKeyArgs {
  LevelCtx x;
  uint32_t items;           // items in this level's concatenated array
  const uint32_t* vals;     // original index per item, or nullptr (level 0)
  uint32_t* vals_out;       // level 0 only: receives the original index per item
  const uint32_t* ranks;    // k * total
  uint32_t total;
  int k, mode;
  const uint8_t* dims;      // split dimension per node (widest mode)
  uint64_t* keys_out;
  uint32_t* hist;           // passes * 256
  int passes;
};
cudaError_t launch_level_keys(const LevelKeyArgs& a, int num_sms, cudaStream_t st);

// Segmented levels: one block per (segment, chunk of kSegChunk items); keys
// are the 32-bit ranks, histograms are per (pass, segment, digit).
constexpr uint32_t kSegChunk = 8192;
struct SegKeyArgs {
  LevelCtx x;
  uint32_t chunks;          // total chunks of the level
  const uint32_t* vals;     // original index per item, or nullptr (level 0)
  uint32_t* vals_out;       // level 0 only
  const uint32_t* ranks;
  uint32_t total;
  int k, mode;
  const uint8_t* dims;
  uint32_t* keys_out;
  uint32_t* seg_hist;       // [passes][nseg][256]
  uint32_t nseg;
  int passes;
};
cudaError_t launch_seg_level_keys(const SegKeyArgs& a, cudaStream_t st);

struct WidestArgs {
  LevelCtx x;              // x.act is the level whose nodes are split
  const unsigned char* pts;
  int k, stride;
  const uint32_t* perm;    // orig index of each pinned node, or nullptr (points in tree order)
  const float* boxes_in;   // per active entry: 2^l boxes of 2k floats
  float* boxes_out;        // per next-level active entry: 2^(l+1) boxes
  uint8_t* dims;           // per node
  uint32_t total_threads;  // nact << l
  float* boxes_local;      // domains of the roots of local subtrees (sets leaving)
  const LocalSet* lsets;   // their slots (nullptr: no local finish)
};
cudaError_t launch_widest_root(const SetInfo* sets, const ActiveEntry* act0, uint32_t nact,
                               const uint32_t* bbox, int k, float* boxes0, uint8_t* dims, int ctype,
                               cudaStream_t st);
cudaError_t launch_widest_children(const WidestArgs& a, cudaStream_t st);
// validator, tight-box rule: per-node subtree boxes (n x 2k keys) and dims
cudaError_t launch_tight_validate_dims(const unsigned char* pts, uint32_t n, int k, int stride,
                                       uint32_t* box, uint8_t* dims, int ctype, cudaStream_t st);
cudaError_t launch_rr_dims(uint8_t* dims, const SetInfo* sets, uint32_t nsets, uint32_t total,
                           int k, int dim0, cudaStream_t st);

// Placement: one cycle leader (and one staged record) per kPermGroup nodes.
constexpr uint32_t kPermGroup = 16;

struct PermuteArgs {
  unsigned char* pts;
  uint32_t total;
  int stride;
  uint32_t* perm;          // node -> original index, marked on the way
  unsigned char* stage;    // ceil(total / kPermGroup) records
  uint32_t* err;
};
cudaError_t launch_permute(const PermuteArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_place_gather(const PermuteArgs& a, unsigned char* tmp, int num_sms, cudaStream_t st);
// Records of stride 4k rebuilt from their entries (input order) if the build
// failed after writing records directly at their nodes.
cudaError_t launch_restore(unsigned char* pts, const uint4* ents, uint32_t total, int k, const uint32_t* err,
                           int ctype, cudaStream_t st);
cudaError_t launch_init_bbox(uint32_t* bbox, uint32_t nsets, int k, cudaStream_t st);
cudaError_t launch_unmark(const uint32_t* perm, int32_t* out, uint32_t total, cudaStream_t st);

cudaError_t launch_validate(const unsigned char* pts, uint32_t n, int k, int stride, int mode,
                            const uint8_t* dims, uint32_t* first_bad, cudaStream_t st);

}  // namespace kdb
