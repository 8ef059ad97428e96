// kdb_api.cu -- host driver of the build and the C ABI declared in kdb.h.
//
// The level loop (Sec. 3.2, parallelKDTreeBuild), k <= 3:
//   prepass       one read of the records: a 16-byte entry per point (the
//                 order-preserving keys of its coordinates and its index), NaN
//                 check, scene boxes (widest mode, Sec. 6);
//   level-0 lists per dimension, a stable LSD radix sort of the entries from
//                 input order (kdb_lists.cu): list d is the order of the
//                 level-0 sort (Sec. 3.1) when d is the split dimension;
//   level l       the pivots of level l at rank ss(lChild) of each segment of
//                 the split dimension's list (Observation 1), then a list
//                 advanced by one to three levels of the tag update
//                 (kdb_part.cu); lists are advanced lazily under round robin;
//   local finish  once every subtree holds at most 2^13 - 1 points, one block
//                 per subtree runs its remaining levels on chip (kdb_local.cu);
//   records       without payload, each record is written at its node from its
//                 entry when the node is pinned; with payload, the records are
//                 gathered by the node -> original index array (one int32 per
//                 point), or permuted in place by it (kdb_set_placement).
// k > 3: coordinate ranks by per-dimension radix sorts, then each level sorts
// (set, subtree, rank in the split dimension) keys with the tag update fused
// into the last pass (kdb_sort.cu); the local finish for k = 4 (its k + 1
// lists fill the shared memory), every level globally for k = 5 .. 8; then the
// placement.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/kdb.h"
#include "kdb_launch.h"
#include "kdb_onesweep.cuh"

namespace kdb {
namespace {

// ---------------------------------------------------------------- faults --
int g_fault = KDB_FAULT_NONE;
int64_t g_fault_arg = 0;
constexpr uint64_t kDefaultWaitNs = 4000000000ull;  // a look-back wait gives up after 4 s

// -------------------------------------------------------------- profiling --
enum Kind {
  K_PREPASS,
  K_RADIX,
  K_RADIX_RANK,
  K_RADIX_UPDATE,
  K_LEVEL_KEYS,
  K_WIDEST,
  K_PLACEMENT,
  K_VALIDATE,
  K_LOCAL,
  K_PARTITION,
  K_PIVOT,
  K_LISTS,
  K_LEAN,
  K_COUNT
};
const char* const kKindName[K_COUNT] = {"prepass",      "radix_pass",  "radix_pass_rank",
                                        "radix_pass_update", "level_keys", "widest_dims",
                                        "placement",    "validate",   "local_finish",
                                        "partition_pass", "pivots",     "build_lists",
                                        "lean_top_levels"};
struct ProfRec {
  int kind;
  double bytes;
  int launches;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_placement{KDB_PLACEMENT_AUTO};
// Tuning: the process-wide setting (tile shapes of the two sort kernels and
// the level-0 digit width), and a table of settings kept per kind of build,
// keyed by (bit length of N, k, record stride, mode argument).  A build takes
// its kind's entry, else the process-wide setting.
std::atomic<int> g_part_shape{0}, g_rec_shape{0}, g_rec_bits{8};
struct TuneEntry {
  int log2n, k, stride, mode;  // the kind
  int part, rec, bits;         // its setting
};
constexpr int kTuneTableMax = 256;
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune_table;

int tune_bucket(uint64_t n) {  // bit length of n
  int b = 0;
  while (n) {
    ++b;
    n >>= 1;
  }
  return b;
}

// The setting a build of this kind takes; *found: whether it came from the table.
TuneEntry tuning_for(uint64_t n, int k, int stride, int mode, bool* found) {
  const int b = tune_bucket(n);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry& e : g_tune_table)
      if (e.log2n == b && e.k == k && e.stride == stride && e.mode == mode) {
        if (found) *found = true;
        return e;
      }
  }
  if (found) *found = false;
  return TuneEntry{b, k, stride, mode, g_part_shape.load(), g_rec_shape.load(), g_rec_bits.load()};
}

// Keep (or replace) the entry of a kind; a full table drops its oldest entry.
void put_tuning_entry(const TuneEntry& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (TuneEntry& e : g_tune_table)
    if (e.log2n == t.log2n && e.k == t.k && e.stride == t.stride && e.mode == t.mode) {
      e = t;
      return;
    }
  if ((int)g_tune_table.size() >= kTuneTableMax) g_tune_table.erase(g_tune_table.begin());  // oldest out
  g_tune_table.push_back(t);
}

struct SmemAttr {
  int dev;
  const void* func;
  size_t bytes;
};
std::mutex g_attr_mu;
std::vector<SmemAttr> g_attr;

cudaEvent_t take_event() {
  cudaEvent_t e = nullptr;
  if (!g_event_pool.empty()) {
    e = g_event_pool.back();
    g_event_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    e = nullptr;
  }
  return e;
}

// Brackets one launcher call: counts its kernel launches and, while
// profiling is on, records an event pair around it on the launch stream.
// timed = false: only counted (a launch inside a phase timed as a whole);
// count = false: only timed (the whole phase, its launches counted inside).
class Prof {
 public:
  Prof(int kind, double bytes, int launches, cudaStream_t st, bool timed = true, bool count = true) : st_(st) {
    if (count) g_launches += launches;
    if (!timed) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    rec_.kind = kind;
    rec_.bytes = bytes;
    rec_.launches = launches;
    rec_.a = take_event();
    rec_.b = take_event();
    if (rec_.a && rec_.b && cudaEventRecord(rec_.a, st_) == cudaSuccess) on_ = true;
  }
  ~Prof() {
    if (!on_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (cudaEventRecord(rec_.b, st_) == cudaSuccess) g_prof.push_back(rec_);
  }

 private:
  cudaStream_t st_;
  ProfRec rec_{};
  bool on_ = false;
};

// ------------------------------------------------------------------ pools --
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
int g_sms[64] = {};

kdb_status device_setup(int* dev, cudaMemPool_t* pool, int* sms) {
  if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= 64) {
    cudaGetLastError();
    return KDB_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[*dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = *dev;
    cudaMemPool_t p;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return KDB_ERR_CUDA;
    }
    uint64_t keep = ~0ull;  // keep freed blocks for the next build
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[*dev] = p;
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, *dev);
    g_sms[*dev] = n > 0 ? n : 1;
  }
  *pool = g_pools[*dev];
  *sms = g_sms[*dev];
  return KDB_OK;
}

kdb_status pool_alloc(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t st) {
  *p = nullptr;
  if (bytes == 0) return KDB_OK;
  if (g_fault == KDB_FAULT_ALLOC) {
    g_fault = KDB_FAULT_NONE;
    return KDB_ERR_OUT_OF_MEMORY;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? KDB_ERR_OUT_OF_MEMORY : KDB_ERR_CUDA;
  }
  return KDB_OK;
}

// ------------------------------------------------------------------- plan --
inline int ceil_div_i(int a, int b) { return (a + b - 1) / b; }
// A level sorts segment by segment when every subtree of every active set
// has at least 2^13 - 1 items (>= one radix tile), i.e. L_b - l - 1 >= 13.
constexpr int kSegMinLog = 13;
static_assert((1 << kSegMinLog) - 1 >= kSegTile, "segments must span a tile");
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Plan {
  std::vector<SetInfo> sets;
  uint32_t total = 0;
  int k = 0, stride = 0, mode = 0;  // mode: the split rule (low byte of the mode argument)
  int ctype = kCoordF32;            // coordinate type (KDB_COORDS_INT32 / UINT32)
  int Lmax = 0;        // most levels of any set
  int rb = 0;          // bits of a rank
  int set_bits = 0;    // bits of a set id in the rank-sort keys (0 for one set)
  int rank_passes = 0;
  bool singletons = false;  // a set of one record (its node is its record)
  bool too_wide = false;    // (set, subtree, rank) needs more than 64 bits
  int mode_arg = 0;     // the mode argument as given (the tuning table's key)
  int part_shape = -1, rec_shape = -1;  // tile shapes; -1: from the tuning (make_plan)
  int rec_bits = -1;                    // level-0 digit width; -1: from the tuning
  int dim0 = 0;              // round robin: level l splits in dimension (l + dim0) mod k
  bool has_domain = false;   // widest extent: the root's domain is given, not the scene box
  float domain[2 * kMaxK] = {};  // its lower corner, then its upper corner
  int placement = -1;                    // -1: the process-wide setting
  std::vector<std::vector<ActiveEntry>> act;  // per level l = 0 .. Lmax-2
  std::vector<uint32_t> items;                // per level
  std::vector<int> passes;                    // per level
  std::vector<uint32_t> box_slots;            // per level (widest)
  std::vector<char> seg;                      // per level: segmented sort (32-bit rank keys)
  std::vector<uint32_t> nseg, chunks;         // per segmented level
  std::vector<size_t> hist_off;               // per level: offset (in u32) into the histograms
  uint32_t max_items = 0, max_boxes = 0;
  int total_passes = 0;

  // workspace layout (byte offsets)
  size_t o_keysA, o_keysB, o_valsA, o_valsB, o_ckeys, o_ranks, o_perm, o_dims, o_boxA, o_boxB,
      o_status, o_hist, o_tickets, o_err, o_bbox, o_stage, o_sets, o_act, bytes;
  std::vector<size_t> act_off;  // element offset of each level's active list in the table
  // local finish (k <= kLocalMaxK): subtrees of <= 2^13 - 1 points run on chip
  bool use_local = false;
  std::vector<LocalSet> lsets;
  std::vector<LocalWork> work;
  uint32_t local_boxes = 0;
  size_t o_vloc, o_lbox, o_lsets, o_work, o_whole;
  // presorted lists (k <= 3): one list of 16-byte entries per dimension
  bool use_lists = false;
  size_t o_rows, o_lists, o_lorig, o_piv, o_l0;
  size_t o_lents = 0;        // list 0 handed to the local finish as entries
  bool has_lents = false;
  bool can_direct = false;   // records (stride 4k) can be written from their entries
  size_t o_gather = 0, gather_bytes = 0;  // placement through spare workspace
  size_t rec_hist_off = 0;  // record-sort histograms (in u32, inside the histogram area)
  // Round robin over one set, k >= 2, at least two global levels: list
  // dim0 + 1 is sorted by (side of the root, key) in its last digit pass and
  // starts on level 1 (8-bit digits; the workspace is sized for it whatever
  // the width).  tag_hist_off: its (side, digit) counts (512 u32).
  bool tag_fold_room = false;
  size_t tag_hist_off = 0;
  bool side_list = false;  // list dim0 + 2 sorted on a second stream (one set, k >= 3)
  int rec_regions = 1;     // look-back regions of the level-0 sorts, tiles * 256 words each
  uint32_t max_nseg = 0;
  uint64_t kstride = 0;  // elements between two dimensions' coordinate keys
};

// Levels run on the whole GPU for set b: all of them (packed keys), or, with
// the local finish, those whose subtrees still hold >= 2^13 - 1 points.
inline int global_levels(const Plan& P, uint32_t n) {
  if (n < 2) return 0;
  const int L = num_levels(n);
  return P.use_local ? std::max(0, L - kLocalLog) : L - 1;
}

void make_plan(Plan& P) {
  if (P.part_shape < 0 || P.rec_shape < 0 || P.rec_bits < 0) {
    const TuneEntry t = tuning_for(P.total, P.k, P.stride, P.mode_arg, nullptr);
    if (P.part_shape < 0) P.part_shape = t.part;
    if (P.rec_shape < 0) P.rec_shape = t.rec;
    if (P.rec_bits < 0) P.rec_bits = t.bits;
  }
  uint32_t nmax = 0;
  for (const SetInfo& s : P.sets) {
    nmax = std::max(nmax, s.n);
    if (s.n == 1) P.singletons = true;
  }
  P.Lmax = nmax ? num_levels(nmax) : 0;
  P.rb = bits_for(nmax);
  const uint32_t ns = (uint32_t)P.sets.size();
  P.set_bits = ns > 1 ? bits_for(ns) : 0;
  P.rank_passes = ceil_div_i(32 + P.set_bits, 8);
  P.use_local = P.k <= kLocalMaxK;
  P.use_lists = P.use_local && P.k <= 3;
  if (P.mode == KDB_SPLIT_WIDEST_TIGHT && !P.use_lists) P.too_wide = true;  // not supported
  int levels = 0;
  for (const SetInfo& si : P.sets) levels = std::max(levels, global_levels(P, si.n));
  if (P.use_local) {
    P.lsets.resize(ns);
    uint32_t lbox = 0;
    for (uint32_t b = 0; b < ns; ++b) {
      const SetInfo& si = P.sets[b];
      LocalSet ls;
      ls.off = si.off;
      ls.n = si.n;
      ls.l0 = global_levels(P, si.n);
      ls.lbox0 = lbox;
      if (si.n >= 2) {
        for (uint32_t r = 0; r < (1u << ls.l0); ++r) P.work.push_back(LocalWork{b, r});
        if (ls.l0 > 0) lbox += 1u << ls.l0;
      }
      P.lsets[b] = ls;
    }
    P.local_boxes = lbox;
  }
  P.act.assign(levels, {});
  P.items.assign(levels, 0);
  P.passes.assign(levels, 0);
  P.box_slots.assign(levels, 0);
  P.seg.assign(levels, 0);
  P.nseg.assign(levels, 0);
  P.chunks.assign(levels, 0);
  P.hist_off.assign(levels, 0);
  // list mode sorts 16-byte entries per set (histograms added below); the
  // other modes rank every dimension first
  size_t hist_words = P.use_lists ? 0 : (size_t)P.k * P.rank_passes * kRadixBins;
  for (int l = 0; l < levels; ++l) {
    uint32_t base = 0;
    bool all_long = true;  // every segment of every active set >= 2^13 - 1 items
    for (uint32_t b = 0; b < ns; ++b) {
      const uint32_t n = P.sets[b].n;
      if (l >= global_levels(P, n)) continue;
      ActiveEntry e;
      e.set = b;
      e.base = base;
      e.next = -1;
      e.box0 = (uint32_t)P.act[l].size() << l;
      e.chunk0 = 0;
      e.cps = 0;
      base += n - full_nodes(l);
      if (num_levels(n) - l - 1 < kSegMinLog) all_long = false;
      P.act[l].push_back(e);
    }
    P.items[l] = base;
    const uint32_t na = (uint32_t)P.act[l].size();
    P.seg[l] = all_long && na > 0 && P.rb <= 32;
    P.hist_off[l] = hist_words;
    P.max_nseg = std::max(P.max_nseg, na << l);
    if (P.use_lists) {
      P.passes[l] = P.k;  // one partition pass per list
      if (l == 0) {       // per-set chunks of the level-0 histograms
        uint32_t chunk = 0;
        for (ActiveEntry& e : P.act[0]) {
          e.chunk0 = chunk;
          e.cps = (P.sets[e.set].n + kSegChunk - 1) / kSegChunk;
          chunk += e.cps;
        }
        P.chunks[0] = chunk;
        P.rec_hist_off = hist_words;  // room for the most passes of any width
        hist_words += (size_t)P.k * kRecMaxPasses * na * kRadixBins;
        P.tag_hist_off = hist_words;
        hist_words += 2 * kRadixBins;
      }
    } else if (P.seg[l]) {
      P.passes[l] = std::max(1, ceil_div_i(P.rb, 8));
      P.nseg[l] = na << l;
      uint32_t chunk = 0;
      for (ActiveEntry& e : P.act[l]) {
        const int h = num_levels(P.sets[e.set].n) - l - 1;
        const uint32_t full = (uint32_t)((1ull << (h + 1)) - 1);
        e.chunk0 = chunk;
        e.cps = (full + kSegChunk - 1) / kSegChunk;
        chunk += e.cps << l;
      }
      P.chunks[l] = chunk;
      hist_words += (size_t)P.passes[l] * P.nseg[l] * kRadixBins;
    } else {
      const int abits = na > 1 ? bits_for(na) : 0;
      if (abits + l + P.rb > 64) P.too_wide = true;  // packed key would not fit 64 bits
      P.passes[l] = std::max(1, ceil_div_i(abits + l + P.rb, 8));
      hist_words += (size_t)P.passes[l] * kRadixBins;
    }
    P.box_slots[l] = na << l;
    P.max_items = std::max(P.max_items, base);
    P.max_boxes = std::max(P.max_boxes, P.box_slots[l]);
    P.total_passes += P.passes[l];
  }
  for (int l = 0; l + 1 < levels; ++l) {
    size_t j = 0;
    for (ActiveEntry& e : P.act[l]) {
      while (j < P.act[l + 1].size() && P.act[l + 1][j].set < e.set) ++j;
      if (j < P.act[l + 1].size() && P.act[l + 1][j].set == e.set) e.next = (int32_t)j;
    }
  }
  P.total_passes += P.k * (P.use_lists ? kRecMaxPasses : P.rank_passes);

  const uint64_t T = P.total;
  const size_t ksz = P.sets.size() > 1 ? 8 : 4;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  // 64-bit keys: several sets' rank sorts, or packed level keys; else 32-bit
  // rank sorts and packed-key levels (not used in list mode)
  const size_t kb = P.use_lists ? 0 : 8;
  P.o_keysA = take(T * kb);
  P.o_keysB = take(T * kb);
  P.o_valsA = take(P.use_lists ? 0 : T * 4);
  P.o_valsB = take(P.use_lists ? 0 : T * 4);
  P.kstride = (T + 63) & ~uint64_t(63);  // per-dimension key arrays start 256-byte aligned
  P.o_ckeys = take(P.use_lists ? 0 : P.kstride * P.k * ksz);
  P.o_ranks = take(P.use_lists ? 0 : T * P.k * 4);
  P.o_perm = take(T * 4);
  P.o_dims = take(T);
  const size_t box_bytes = P.mode == KDB_SPLIT_WIDEST_EXTENT ? (size_t)P.max_boxes * 2 * P.k * 4 : 0;
  P.o_boxA = take(box_bytes);
  P.o_boxB = take(box_bytes);
  // look-back words: 256 per tile of the radix passes (the smallest of their
  // tiles), kLiftBins per partition tile
  const uint64_t min_tile =
      std::min<uint64_t>(std::min(kSortTile, kSegTile), (uint64_t)rec_sort_tile());
  const size_t tiles = (std::max<uint64_t>(T, P.max_items) + min_tile - 1) / min_tile;
  const size_t part_tiles = (std::max<uint64_t>(T, P.max_items) + kPartTile - 1) / kPartTile;
  P.tag_fold_room = P.use_lists && P.mode == KDB_SPLIT_ROUND_ROBIN && P.sets.size() == 1 && P.k >= 2 &&
                    levels >= 2;
  // one set, k = 3: list dim0 + 2 is sorted on a second stream beside the
  // others, with look-back words of its own
  P.side_list = P.use_lists && P.sets.size() == 1 && P.k >= 3 && levels >= 1;
  // regions of look-back words for the level-0 sorts: the tagged pass takes
  // a second (one per side), the side stream's passes a third
  P.rec_regions = (P.side_list ? P.k : 1) + (P.tag_fold_room ? 1 : 0);
  P.o_status = take(std::max(tiles * kRadixBins * P.rec_regions, part_tiles * kLiftBins) * 8);
  P.o_hist = take(hist_words * 4);
  P.o_tickets = take((size_t)P.total_passes * 4);
  P.o_err = take(4);
  P.o_bbox = take(P.sets.size() * 2 * P.k * 4);
  P.o_stage = take(((T + kPermGroup - 1) / kPermGroup) * (size_t)P.stride);
  P.o_sets = take(P.sets.size() * sizeof(SetInfo));
  size_t nact = 0;
  P.act_off.assign(levels, 0);
  for (int l = 0; l < levels; ++l) {
    P.act_off[l] = nact;
    nact += P.act[l].size();
  }
  P.o_act = take(std::max<size_t>(nact, 1) * sizeof(ActiveEntry));
  P.o_vloc = take(P.use_local && !P.use_lists ? T * 4 : 0);
  P.o_lbox = take(P.use_local && P.mode == KDB_SPLIT_WIDEST_EXTENT
                      ? (size_t)P.local_boxes * 2 * P.k * 4 : 0);
  P.o_lsets = take(P.lsets.size() * sizeof(LocalSet));
  P.o_work = take(P.work.size() * sizeof(LocalWork));
  P.o_whole = take(sizeof(ActiveEntry));  // one segment spanning the whole array
  const bool L = P.use_lists, G = L && levels > 0;  // G: there are global levels
  P.o_rows = take(L ? T * 16 : 0);                   // entries in input order
  P.o_lists = take(G ? T * 16 * 2 * P.k : 0);        // per dimension, double-buffered
  P.o_lorig = take(G ? T * 4 * P.k : 0);             // lists handed to the local finish
  P.o_piv = take(L ? (size_t)kLiftMax * std::max<uint32_t>(P.max_nseg, 1) * 8 : 0);  // last 3 levels
  P.o_l0 = take(G && P.sets.size() > 1 ? T * 16 : 0);  // level-0 array of several sets
  P.can_direct = L && P.stride == 4 * P.k;
  // list 0 handed over as entries: records written from them (stride 4k),
  // and the keys of the tight-box rule in the local finish
  P.has_lents = (P.can_direct || P.mode == KDB_SPLIT_WIDEST_TIGHT) && G;
  P.o_lents = take(P.has_lents ? T * 16 : 0);
  P.bytes = o;
  // workspace that is dead once the local finish has run, one contiguous
  // range: the placement may gather the records into it
  P.o_gather = L ? P.o_rows : P.o_keysA;
  P.gather_bytes = (L ? P.o_piv : P.o_perm) - P.o_gather;
}

kdb_status check_common(int64_t n, int k, int stride) {
  if (n < 0 || n > 2147483647LL) return KDB_ERR_INVALID_ARGUMENT;
  if (k < 1 || k > kMaxK) return KDB_ERR_INVALID_ARGUMENT;
  if (stride < 4 * k || stride % 4 != 0) return KDB_ERR_INVALID_ARGUMENT;
  return KDB_OK;
}

// The mode argument: a split rule in the low byte, optionally OR'ed with one
// of KDB_COORDS_INT32 / KDB_COORDS_UINT32.
kdb_status check_mode(kdb_split_mode mode) {
  const int m = (int)mode;
  if (m & ~(0xFF | KDB_COORDS_INT32 | KDB_COORDS_UINT32)) return KDB_ERR_INVALID_ARGUMENT;
  if ((m & KDB_COORDS_INT32) && (m & KDB_COORDS_UINT32)) return KDB_ERR_INVALID_ARGUMENT;
  const int split = m & 0xFF;
  if (split != KDB_SPLIT_ROUND_ROBIN && split != KDB_SPLIT_WIDEST_EXTENT &&
      split != KDB_SPLIT_WIDEST_TIGHT)
    return KDB_ERR_INVALID_ARGUMENT;
  // the clipped-domain rule clips float boxes: float32 coordinates only
  if ((m & (KDB_COORDS_INT32 | KDB_COORDS_UINT32)) && split == KDB_SPLIT_WIDEST_EXTENT)
    return KDB_ERR_INVALID_ARGUMENT;
  return KDB_OK;
}
// The tight-box rule runs on the presorted lists only (k <= 3).
kdb_status check_mode_k(kdb_split_mode mode, int k) {
  if (check_mode(mode) != KDB_OK) return KDB_ERR_INVALID_ARGUMENT;
  return ((int)mode & 0xFF) == KDB_SPLIT_WIDEST_TIGHT && k > 3 ? KDB_ERR_INVALID_ARGUMENT : KDB_OK;
}
inline int split_of(int mode) { return mode & 0xFF; }
inline int ctype_of(int mode) {
  return (mode & KDB_COORDS_INT32) ? kCoordI32 : ((mode & KDB_COORDS_UINT32) ? kCoordU32 : kCoordF32);
}

#define KDB_CK(call)                      \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      cudaGetLastError();                 \
      return KDB_ERR_CUDA;                \
    }                                     \
  } while (0)

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + off);
}

// Copies the plan's tables (sets, active lists, local work) into the
// workspace; with sync, from the host synchronously (plans made once).
kdb_status upload_tables(const Plan& P, void* ws, cudaStream_t st, bool sync) {
  auto copy = [&](void* dst, const void* src, size_t bytes) {
    return sync ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice)
                : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  KDB_CK(copy(at<SetInfo>(ws, P.o_sets), P.sets.data(), P.sets.size() * sizeof(SetInfo)));
  std::vector<ActiveEntry> flat;
  for (const auto& v : P.act) flat.insert(flat.end(), v.begin(), v.end());
  if (!flat.empty())
    KDB_CK(copy(at<ActiveEntry>(ws, P.o_act), flat.data(), flat.size() * sizeof(ActiveEntry)));
  // pageable sources: each copy has completed when the call returns
  if (P.use_local) {
    KDB_CK(copy(at<LocalSet>(ws, P.o_lsets), P.lsets.data(), P.lsets.size() * sizeof(LocalSet)));
    if (!P.work.empty())
      KDB_CK(copy(at<LocalWork>(ws, P.o_work), P.work.data(), P.work.size() * sizeof(LocalWork)));
  }
  ActiveEntry w{};
  w.set = 0;
  w.base = 0;
  w.next = -1;
  KDB_CK(copy(at<ActiveEntry>(ws, P.o_whole), &w, sizeof w));
  return KDB_OK;
}

// The plan's tables as one host image of the workspace span [*off, *off +
// *bytes) that holds them (gaps zero); false where that span also holds
// large work arrays (the packed-key path), which upload_tables copies
// table by table instead.
bool table_image_span(const Plan& P, size_t* off, size_t* bytes) {
  const size_t b = P.o_sets, e = align256(P.o_whole + sizeof(ActiveEntry));
  if (P.o_lbox - P.o_vloc > ((size_t)1 << 16) || P.o_lsets - P.o_lbox > ((size_t)1 << 20)) return false;
  *off = b;
  *bytes = e - b;
  return true;
}
void fill_table_image(const Plan& P, unsigned char* img, size_t off) {
  auto put = [&](size_t o, const void* src, size_t n) {
    if (n) std::memcpy(img + (o - off), src, n);
  };
  put(P.o_sets, P.sets.data(), P.sets.size() * sizeof(SetInfo));
  size_t at_act = P.o_act;
  for (const auto& v : P.act) {
    put(at_act, v.data(), v.size() * sizeof(ActiveEntry));
    at_act += v.size() * sizeof(ActiveEntry);
  }
  if (P.use_local) {
    put(P.o_lsets, P.lsets.data(), P.lsets.size() * sizeof(LocalSet));
    put(P.o_work, P.work.data(), P.work.size() * sizeof(LocalWork));
  }
  ActiveEntry w{};
  w.set = 0;
  w.base = 0;
  w.next = -1;
  put(P.o_whole, &w, sizeof w);
}

// Plans of single builds, kept for builds of the same kind: the same N, k,
// stride, mode argument and tuning setting give the same plan, so a repeated
// build skips the planning and uploads its tables from pinned host memory in
// one asynchronous copy.  A few recent kinds are kept; an entry stays alive
// while a call that took it runs.
struct CachedPlan {
  Plan P;
  unsigned char* h_img = nullptr;  // pinned, or nullptr: tables uploaded one by one
  size_t img_off = 0, img_bytes = 0;
  ~CachedPlan() {
    if (h_img) cudaFreeHost(h_img);
  }
};
struct PlanKey {
  uint32_t n;
  int k, stride, mode_arg, part, rec, bits;
  bool operator==(const PlanKey& o) const {
    return n == o.n && k == o.k && stride == o.stride && mode_arg == o.mode_arg && part == o.part &&
           rec == o.rec && bits == o.bits;
  }
};
constexpr size_t kPlanCacheMax = 8;
std::mutex g_pcache_mu;
// never destroyed: its pinned images may outlive the CUDA runtime at exit
auto* g_pcache = new std::vector<std::pair<PlanKey, std::shared_ptr<CachedPlan>>>();

std::shared_ptr<CachedPlan> cached_plan(int64_t n, int k, int stride, int mode_arg) {
  const TuneEntry t = tuning_for((uint64_t)n, k, stride, mode_arg, nullptr);
  const PlanKey key{(uint32_t)n, k, stride, mode_arg, t.part, t.rec, t.bits};
  {
    std::lock_guard<std::mutex> lk(g_pcache_mu);
    for (size_t i = 0; i < g_pcache->size(); ++i)
      if ((*g_pcache)[i].first == key) {
        auto e = (*g_pcache)[i];
        g_pcache->erase(g_pcache->begin() + i);
        g_pcache->push_back(e);  // most recent last
        return e.second;
      }
  }
  auto cp = std::make_shared<CachedPlan>();
  Plan& P = cp->P;
  P.sets.push_back(SetInfo{0u, (uint32_t)n});
  P.total = (uint32_t)n;
  P.k = k;
  P.stride = stride;
  P.mode = mode_arg & 0xFF;
  P.ctype = ctype_of(mode_arg);
  P.mode_arg = mode_arg;
  P.part_shape = t.part;
  P.rec_shape = t.rec;
  P.rec_bits = t.bits;
  make_plan(P);
  if (!P.too_wide && table_image_span(P, &cp->img_off, &cp->img_bytes)) {
    void* h = nullptr;
    if (cudaHostAlloc(&h, cp->img_bytes, cudaHostAllocDefault) == cudaSuccess) {
      cp->h_img = static_cast<unsigned char*>(h);
      std::memset(cp->h_img, 0, cp->img_bytes);
      fill_table_image(P, cp->h_img, cp->img_off);
    } else {
      cudaGetLastError();
    }
  }
  std::lock_guard<std::mutex> lk(g_pcache_mu);
  if (g_pcache->size() >= kPlanCacheMax) g_pcache->erase(g_pcache->begin());
  g_pcache->push_back({key, cp});
  return cp;
}

// Enqueues the whole build on `st`.  Does not synchronise.  With
// tables_ready the plan's tables are already in the workspace: then only
// kernels and memsets are enqueued (no host memory is read), so the call can
// be captured into a CUDA graph.
// Records that arrive from host memory during the build: chunk c is copied
// to the device on stream `cs` and event ev[c] marks its arrival.
struct HostFeed {
  const unsigned char* h = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[8] = {};
  int chunks = 0;
};

// A second stream for work that may run beside `st`: fork() makes it wait
// for what `st` has enqueued so far, join() marks the end of its work, and
// wait() makes `st` wait for that.  The stream and events are released when
// the object goes (after their work, by the runtime's deferred release).
struct SideStream {
  cudaStream_t s = nullptr, st0 = nullptr;
  cudaEvent_t f = nullptr, j = nullptr;
  bool joined = false, waited = false;
  cudaError_t fork(cudaStream_t st) {
    st0 = st;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(f, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, f, 0);
    return e;
  }
  cudaError_t join(cudaStream_t) {
    joined = true;
    return cudaEventRecord(j, s);
  }
  cudaError_t wait(cudaStream_t st) {
    waited = true;
    return cudaStreamWaitEvent(st, j, 0);
  }
  ~SideStream() {
    // a build left early: `st` still waits for the side stream's work, so
    // that nothing freed in stream order on `st` is in use there
    if (s && j && !waited) {
      if (!joined) cudaEventRecord(j, s);
      cudaStreamWaitEvent(st0, j, 0);
    }
    if (f) cudaEventDestroy(f);
    if (j) cudaEventDestroy(j);
    if (s) cudaStreamDestroy(s);
  }
};

kdb_status enqueue_build(const Plan& P, unsigned char* pts, void* ws, int sms,
                         int32_t* out_orig, uint8_t* out_dim, cudaStream_t st,
                         bool tables_ready = false, const HostFeed* feed = nullptr) {
  const uint32_t T = P.total;
  const int k = P.k;
  const int part_shape = P.part_shape;
  const int rec_shape = P.rec_shape;
  const int rec_bits = P.rec_bits;
  const int rec_np = rec_passes(rec_bits);
  uint64_t* keysA = at<uint64_t>(ws, P.o_keysA);
  uint64_t* keysB = at<uint64_t>(ws, P.o_keysB);
  uint32_t* valsA = at<uint32_t>(ws, P.o_valsA);
  uint32_t* valsB = at<uint32_t>(ws, P.o_valsB);
  uint32_t* ranks = at<uint32_t>(ws, P.o_ranks);
  uint32_t* perm = at<uint32_t>(ws, P.o_perm);
  uint8_t* dims = at<uint8_t>(ws, P.o_dims);
  float* boxA = at<float>(ws, P.o_boxA);
  float* boxB = at<float>(ws, P.o_boxB);
  uint64_t* status = at<uint64_t>(ws, P.o_status);
  uint32_t* hist = at<uint32_t>(ws, P.o_hist);
  uint32_t* tickets = at<uint32_t>(ws, P.o_tickets);
  uint32_t* err = at<uint32_t>(ws, P.o_err);
  uint32_t* bbox = at<uint32_t>(ws, P.o_bbox);
  SetInfo* d_sets = at<SetInfo>(ws, P.o_sets);
  ActiveEntry* d_act = at<ActiveEntry>(ws, P.o_act);
  const bool multi = P.sets.size() > 1;
  const bool widest = P.mode == KDB_SPLIT_WIDEST_EXTENT;
  const bool tight = P.mode == KDB_SPLIT_WIDEST_TIGHT;
  const bool bydim = widest || tight;  // split dimension stored per node

  // tables and zeroed state: look-back words, histograms, tickets, error word
  if (!tables_ready) {
    kdb_status s = upload_tables(P, ws, st, false);
    if (s != KDB_OK) return s;
  }
  uint32_t* vals_local = at<uint32_t>(ws, P.o_vloc);
  float* boxes_local = at<float>(ws, P.o_lbox);
  LocalSet* d_lsets = at<LocalSet>(ws, P.o_lsets);
  LocalWork* d_work = at<LocalWork>(ws, P.o_work);
  ActiveEntry* d_whole = at<ActiveEntry>(ws, P.o_whole);
  KDB_CK(cudaMemsetAsync(status, 0, P.o_hist - P.o_status, st));
  KDB_CK(cudaMemsetAsync(hist, 0, P.o_bbox - P.o_hist, st));  // hist, tickets, err
  if (bydim) KDB_CK(launch_init_bbox(bbox, (uint32_t)P.sets.size(), k, st));
  if (out_dim || bydim) KDB_CK(cudaMemsetAsync(dims, 0, T, st));

  const uint64_t wait_ns =
      (g_fault == KDB_FAULT_LOOKBACK || g_fault == KDB_FAULT_LOOKBACK_PARTITION)
          ? (uint64_t)std::max<int64_t>(g_fault_arg, 1) * 1000ull
          : kDefaultWaitNs;
  const bool fault_lb = g_fault == KDB_FAULT_LOOKBACK;
  const bool fault_part = g_fault == KDB_FAULT_LOOKBACK_PARTITION;
  if (fault_lb || fault_part) g_fault = KDB_FAULT_NONE;
  int g = 0;  // pass counter within the build
  auto ctl = [&](uint32_t n, int shift, const uint32_t* h) {
    PassCtl c{};
    c.n = n;
    c.shift = shift;
    c.hist = h;
    c.status = status;
    c.ticket = tickets + g;
    c.epoch = (uint32_t)(g + 1);
    c.wait_epoch = fault_lb ? (uint32_t)(g + 1) + 0x10000000u : c.epoch;
    c.wait_ns = wait_ns;
    c.err = err;
    c.status_words = (P.o_hist - P.o_status) / 8;
    ++g;
    return c;
  };

  // ---- prepass
  PrepassArgs pa{};
  pa.pts = pts;
  pa.total = T;
  pa.k = k;
  pa.stride = P.stride;
  pa.sets = d_sets;
  pa.nsets = (uint32_t)P.sets.size();
  uint4* ents0 = at<uint4>(ws, P.o_rows);
  if (P.use_lists) {
    pa.ents = ents0;
  } else {
    pa.keys32 = multi ? nullptr : at<uint32_t>(ws, P.o_ckeys);
    pa.keys64 = multi ? at<uint64_t>(ws, P.o_ckeys) : nullptr;
    pa.kstride = P.kstride;
    pa.hist = hist;
    pa.passes = P.rank_passes;
  }
  pa.bbox = bydim ? bbox : nullptr;  // the root's domain and its tight box alike
  pa.err = err;
  pa.ctype = P.ctype;
  // one set on the list path: the vectorised prepass also counts the level-0
  // sort's digit histograms, so that the entries are not read again for them
  const bool hist_in_prepass = P.use_lists && !multi && !P.act.empty() && !P.act[0].empty() &&
                               prepass_fuses_rec_hist(pa);
  if (hist_in_prepass) {
    pa.rec_hist = hist + P.rec_hist_off;
    pa.rec_bits = rec_bits;
  }
  {
    Prof pf(K_PREPASS, P.use_lists ? (double)T * (4.0 * k + 16.0) : (double)T * k * (4.0 + (multi ? 8 : 4)),
            feed ? feed->chunks : 1, st);
    if (!feed) {
      KDB_CK(launch_prepass(pa, sms, st));
    } else {
      // the records come from host memory in chunks: the copy of chunk c + 1
      // (on the feed's stream) overlaps the prepass of chunk c
      for (int c = 0; c < feed->chunks; ++c) {
        const uint32_t b = (uint32_t)((uint64_t)T * c / feed->chunks);
        const uint32_t e = (uint32_t)((uint64_t)T * (c + 1) / feed->chunks);
        KDB_CK(cudaMemcpyAsync(pts + (size_t)b * P.stride, feed->h + (size_t)b * P.stride,
                               (size_t)(e - b) * P.stride, cudaMemcpyHostToDevice, feed->cs));
        KDB_CK(cudaEventRecord(feed->ev[c], feed->cs));
      }
      for (int c = 0; c < feed->chunks; ++c) {
        pa.beg = (uint32_t)((uint64_t)T * c / feed->chunks);
        pa.end = (uint32_t)((uint64_t)T * (c + 1) / feed->chunks);
        KDB_CK(cudaStreamWaitEvent(st, feed->ev[c], 0));
        if (pa.end > pa.beg) KDB_CK(launch_prepass(pa, sms, st));
      }
      pa.beg = pa.end = 0;
    }
  }
  if (P.has_domain && bydim) {
    // the root's domain is given (a subtree of a larger tree): it replaces
    // the scene box as the root's domain, stored as coordinate keys
    uint32_t keys[2 * kMaxK];
    for (int d = 0; d < 2 * k; ++d) {
      uint32_t bits;
      std::memcpy(&bits, &P.domain[d < k ? d : kMaxK + d - k], 4);
      keys[d] = float_key(bits);
    }
    KDB_CK(cudaMemcpyAsync(bbox, keys, 2 * k * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  }
  uint32_t* hcur = hist + (size_t)k * P.rank_passes * kRadixBins;

  // ---- per-dimension ranks (packed-key levels, k >= 4)
  auto rank_out = [&](int d) {
    RankOut o{};
    o.d = d;
    o.rank = ranks + (size_t)d * T;
    return o;
  };
  for (int d = 0; d < (P.use_lists ? 0 : k); ++d) {
    const uint32_t* hd = hist + (size_t)d * P.rank_passes * kRadixBins;
    if (!multi) {
      // one set: the segmented pass with a single segment spanning the array
      LevelCtx wx{};
      wx.sets = d_sets;
      wx.act = d_whole;
      wx.nact = 1;
      wx.l = 0;
      wx.dim0 = P.dim0;
      wx.err = err;
      const uint32_t* kin = at<uint32_t>(ws, P.o_ckeys) + (size_t)d * P.kstride;
      const uint32_t* vin = nullptr;
      uint32_t* kb[2] = {reinterpret_cast<uint32_t*>(keysA), reinterpret_cast<uint32_t*>(keysB)};
      uint32_t* vb[2] = {valsA, valsB};
      for (int p = 0; p < P.rank_passes; ++p) {
        PassCtl c = ctl(T, 8 * p, nullptr);
        const uint32_t* hp = hd + p * kRadixBins;
        if (p + 1 == P.rank_passes) {
          Prof pf(K_RADIX_RANK, (double)T * 12, 1, st);
          KDB_CK(seg_pass_rank(kin, vin, wx, hp, rank_out(d), c, st));
        } else {
          Prof pf(K_RADIX, (double)T * 16, 1, st);
          KDB_CK(seg_pass_pingpong(kin, vin, kb[p & 1], vb[p & 1], wx, hp, c, st));
          kin = kb[p & 1];
          vin = vb[p & 1];
        }
      }
    } else {
      const uint64_t* kin = at<uint64_t>(ws, P.o_ckeys) + (size_t)d * P.kstride;
      const uint32_t* vin = nullptr;
      uint64_t* kb[2] = {keysA, keysB};
      uint32_t* vb[2] = {valsA, valsB};
      for (int p = 0; p < P.rank_passes; ++p) {
        PassCtl c = ctl(T, 8 * p, hd + p * kRadixBins);
        if (p + 1 == P.rank_passes) {
          Prof pf(K_RADIX_RANK, (double)T * 16, 1, st);
          KDB_CK(pass_u64_rank(kin, vin, rank_out(d), d_sets, 32, c, st));
        } else {
          Prof pf(K_RADIX, (double)T * 24, 1, st);
          KDB_CK(pass_u64_pingpong(kin, vin, kb[p & 1], vb[p & 1], c, st));
          kin = kb[p & 1];
          vin = vb[p & 1];
        }
      }
    }
  }

  if (P.singletons) {
    // a one-record set is already its own tree: identity entries in perm
    // (every other entry is written by the level loop)
    std::vector<uint32_t> ids;
    for (const SetInfo& s : P.sets)
      if (s.n == 1) ids.push_back(s.off);
    // few and small: write them one by one from a host table
    for (uint32_t id : ids) KDB_CK(cudaMemcpyAsync(perm + id, &id, 4, cudaMemcpyHostToDevice, st));
  }

  // ---- level loop
  const int levels = (int)P.act.size();
  if (bydim && levels > 0)
  {
    Prof pf(K_WIDEST, 0.0, 1, st);
    KDB_CK(launch_widest_root(d_sets, d_act + P.act_off[0], (uint32_t)P.act[0].size(), bbox, k,
                              widest ? boxA : nullptr, dims, P.ctype, st));
  }
  const uint32_t* vals_cur = nullptr;  // level 0: original order
  uint4* lcur[3] = {nullptr, nullptr, nullptr};
  uint4* lnext[3] = {nullptr, nullptr, nullptr};
  uint32_t* lorig = at<uint32_t>(ws, P.o_lorig);
  // pivots of the last kLiftMax levels, level q in slot q % kLiftMax
  uint2* piv_ring[kLiftMax];
  for (int i = 0; i < kLiftMax; ++i)
    piv_ring[i] = at<uint2>(ws, P.o_piv) + (size_t)i * std::max<uint32_t>(P.max_nseg, 1);
  // Round robin: a list is read only on the levels that split in its
  // dimension (the same levels in every set), so it is advanced lazily,
  // several levels in one pass, just before those levels (lat[d]: the level
  // list d is sorted for); a set that leaves the active list within such a
  // pass is handed to the local finish at the level where it leaves.
  const bool lazy = P.use_lists && P.mode == KDB_SPLIT_ROUND_ROBIN;
  // Records without payload are written straight to their nodes from the
  // entries (which hold every coordinate bit) as the nodes are pinned; the
  // caller's array is not read after the prepass, and no placement is left.
  const int placement = P.placement >= 0 ? P.placement : g_placement.load();
  const bool direct = P.can_direct && placement == KDB_PLACEMENT_AUTO;
  uint4* lents = P.has_lents && (direct || tight) ? at<uint4>(ws, P.o_lents) : nullptr;
  int lat[3] = {0, 0, 0};
  auto level_ctx = [&](int l) {
    LevelCtx x{};
    x.sets = d_sets;
    x.act = d_act + P.act_off[l];
    x.act_next = l + 1 < levels ? d_act + P.act_off[l + 1] : nullptr;
    x.nact = (uint32_t)P.act[l].size();
    x.l = l;
    x.dim0 = P.dim0;
    x.rb = P.rb;
    x.err = err;
    x.local_next = P.use_local ? 1 : 0;
    x.vals_local = vals_local;
    return x;
  };
  // advance list d from level p to level q (the local finish's level if
  // handoff), with the pivots of levels p .. q-1
  // (ls, soff, swords: the stream, and the look-back words, of a lift that
  // runs beside others; timed: whether its own time is recorded)
  auto lift = [&](int d, int p, int q, bool handoff, cudaStream_t ls = nullptr, uint64_t soff = 0,
                  uint64_t swords = 0, bool timed = true) -> cudaError_t {
    if (!ls) ls = st;
    PassCtl c = ctl(P.items[p], 0, nullptr);
    if (swords) {
      c.status += soff;
      c.status_words = swords;
    }
    if (fault_part) c.wait_epoch = c.epoch + 0x10000000u;
    PartArgs pa{};
    pa.x = level_ctx(p);
    pa.act_out = q < levels ? d_act + P.act_off[q] : nullptr;
    for (int j = 0; j < kLiftMax - 1; ++j)
      pa.act_mid[j] = p + 1 + j < levels ? d_act + P.act_off[p + 1 + j] : nullptr;
    pa.b = q - p;
    pa.handoff = handoff ? 1 : 0;
    pa.in = lcur[d];
    pa.out_next = lnext[d];
    pa.out_lorig = lorig;
    pa.out_lents = lents;
    for (int e = 0; e < q - p; ++e) pa.piv[e] = piv_ring[(p + e) % kLiftMax];
    pa.dims = dims;
    pa.k = k;
    pa.mode = P.mode;
    pa.dlist = d;
    pa.pos_first = P.mode == KDB_SPLIT_ROUND_ROBIN && (p + P.dim0) % k == d ? 1 : 0;
    pa.n = P.items[p];
    pa.next_items = q < levels ? P.items[q] : 0;
    pa.total = T;
    pa.status = c.status;
    pa.ticket = c.ticket;
    pa.epoch = c.epoch;
    pa.wait_epoch = c.wait_epoch;
    pa.wait_ns = c.wait_ns;
    pa.status_words = c.status_words;
    if (P.sets.size() == 1) {
      pa.single = 1;
      pa.set0 = P.sets[0];
      pa.act0 = P.act[p][0];
      pa.out_base0 = q < levels ? P.act[q][0].base : 0u;
    }
    // algorithmic bytes: every item of level p read once; the survivors
    // written as entries, or (hand-over) as original indices, list 0 as
    // entries when it is handed over whole
    const double wbytes = !handoff ? 16.0 : (lents && d == 0 ? 16.0 : 4.0);
    Prof pf(K_PARTITION, (double)P.items[p] * (16.0 + wbytes), 1, ls, timed);
    pa.shape = part_shape;
    cudaError_t e = launch_partition(pa, ls);
    std::swap(lcur[d], lnext[d]);
    lat[d] = q;
    return e;
  };
  // pivots of level l (Observation 1), from the list of its split dimension
  auto pivots_of = [&](int l, bool timed = true) -> cudaError_t {
    PivotArgs pv{};
    pv.x = level_ctx(l);
    for (int d = 0; d < k; ++d) pv.lists[d] = lcur[d];
    pv.items = P.items[l];
    pv.piv = piv_ring[l % kLiftMax];
    pv.perm = perm;
    pv.dims = dims;
    pv.k = k;
    pv.mode = P.mode;
    pv.pts_out = direct ? pts : nullptr;
    pv.stride = P.stride;
    pv.ctype = P.ctype;
    Prof pf(K_PIVOT, (double)(pv.x.nact << l) * 20, 1, st, timed);
    return launch_pivots(pv, st);
  };
  // list dim0 + 1 arrives on level 1 from its last digit pass (one set,
  // round robin, 8-bit digits): no partition pass for level 1
  const bool fold = P.tag_fold_room && lazy && rec_bits == 8;
  if (P.use_lists) {
    for (int d = 0; d < k; ++d) {
      lcur[d] = at<uint4>(ws, P.o_lists) + (size_t)(2 * d) * T;
      lnext[d] = at<uint4>(ws, P.o_lists) + (size_t)(2 * d + 1) * T;
    }
    if (levels > 0) {
      // level-0 lists: per dimension a stable LSD radix sort of the entries
      // by the coordinate key, from input order (so ties keep index order)
      LevelCtx x0{};
      x0.sets = d_sets;
      x0.act = d_act + P.act_off[0];
      x0.nact = (uint32_t)P.act[0].size();
      x0.l = 0;
      x0.dim0 = P.dim0;
      x0.err = err;
      const uint32_t n0 = P.items[0];
      const uint4* l0 = ents0;
      if (multi) {
        ListBuildArgs lb{};
        lb.x = x0;
        lb.items = n0;
        lb.ents = ents0;
        lb.out = at<uint4>(ws, P.o_l0);
        lb.total = T;
        Prof pf(K_LISTS, (double)n0 * 32, 1, st);
        KDB_CK(launch_gather_level0(lb, st));
        l0 = lb.out;
      }
      RecHistArgs rh{};
      rh.x = x0;
      rh.chunks = P.chunks[0];
      rh.ents = l0;
      rh.hist = hist + P.rec_hist_off;
      rh.nseg = x0.nact;
      rh.k = k;
      rh.bits = rec_bits;
      if (!hist_in_prepass) {
        Prof pf(K_LISTS, (double)n0 * 16, 1, st);
        KDB_CK(launch_rec_hist(rh, st));
      }
      const int d0 = P.dim0 % k, d1 = (P.dim0 + 1) % k;
      uint32_t* thist = hist + P.tag_hist_off;
      // One set, k = 3, `st` not being captured into a graph: every list is
      // sorted on a stream of its own (lists dim0 + 1 and dim0 + 2 on side
      // streams forked from `st`, joined back before the levels), so that
      // their passes run side by side (each pass is bound by its own latency,
      // not by bandwidth); list dim0 + 1 waits for the root's pivot only
      // before the passes that need it.  Look-back regions: one per list,
      // and one more for the right side of the tagged pass.
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      if (P.side_list) KDB_CK(cudaStreamIsCapturing(st, &cap));
      const bool side = P.side_list && cap == cudaStreamCaptureStatusNone;
      const uint64_t region = (P.o_hist - P.o_status) / 8 / P.rec_regions;  // look-back words of one region
      // the passes run side by side, so the phase is timed as a whole
      Prof phase(K_RADIX, (double)n0 * 32 * rec_np * k, rec_np * k, st, side, false);
      SideStream aux[2];
      cudaEvent_t root_done = nullptr;  // the root's pivot is taken
      struct EventGuard {
        cudaEvent_t* e;
        ~EventGuard() {
          if (*e) cudaEventDestroy(*e);
        }
      } root_guard{&root_done};
      // passes [pa, pb) of list d on stream ls with look-back region reg
      auto sort_list = [&](int d, int pa, int pb, cudaStream_t ls, int reg) -> cudaError_t {
        const bool tagged = fold && d == d1;
        for (int p = pa; p < pb; ++p) {
          const uint4* in = p == 0 ? l0 : (((rec_np - p) & 1) ? lnext[d] : lcur[d]);
          // ping-pong between the dimension's two list buffers, ending in lcur
          uint4* out = ((rec_np - 1 - p) & 1) ? lnext[d] : lcur[d];
          PassCtl c = ctl(n0, rec_bits * p, nullptr);
          c.status += (uint64_t)reg * region;
          c.status_words = region;
          const uint32_t* sh = rh.hist + ((size_t)(d * rec_np + p) * x0.nact) * kRadixBins;
          Prof pf(K_RADIX, (double)n0 * 32, 1, ls, !side);
          cudaError_t e;
          if (tagged && p + 1 == rec_np) {
            // the last digit with the side of the root: the list leaves on
            // level 1 (the last region holds the right side's words)
            PassCtl c1 = c;
            c1.status = status + (uint64_t)(P.rec_regions - 1) * region;
            e = launch_rec_tag_pass(in, out, c, c1, piv_ring[0], d0, thist, d, rec_shape, ls);
          } else if (tagged && p + 2 == rec_np) {
            // counts (side of the root, last digit) for the tagged pass
            const RecCount rc{piv_ring[0], d0, thist, rec_bits * (rec_np - 1)};
            e = launch_rec_sort_pass(in, out, c, x0, sh, d, rec_shape, rec_bits, ls, &rc);
          } else {
            e = launch_rec_sort_pass(in, out, c, x0, sh, d, rec_shape, rec_bits, ls);
          }
          if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
      };
      // the passes of list d1 that need the root's pivot: its last two
      const int np_free = fold ? rec_np - 2 : rec_np;
      if (side) {
        for (int j = 0; j < 2; ++j) KDB_CK(aux[j].fork(st));
        KDB_CK(sort_list((P.dim0 + 2) % k, 0, rec_np, aux[1].s, 2));
        KDB_CK(sort_list(d1, 0, np_free, aux[0].s, 1));
        KDB_CK(sort_list(d0, 0, rec_np, st, 0));
        if (fold) {
          KDB_CK(pivots_of(0, false));  // the root (timed with the phase)
          KDB_CK(cudaEventCreateWithFlags(&root_done, cudaEventDisableTiming));
          KDB_CK(cudaEventRecord(root_done, st));
          KDB_CK(cudaStreamWaitEvent(aux[0].s, root_done, 0));
          KDB_CK(sort_list(d1, np_free, rec_np, aux[0].s, 1));
        }
        for (int j = 0; j < 2; ++j) {
          KDB_CK(aux[j].join(st));
          KDB_CK(aux[j].wait(st));
        }
      } else {
        for (int di = 0; di < k; ++di) {
          const int d = (P.dim0 + di) % k;
          KDB_CK(sort_list(d, 0, rec_np, st, 0));
          if (fold && d == d0) KDB_CK(pivots_of(0));  // the root, before list d1's passes need its side
        }
      }
      if (fold) lat[d1] = 1;
    }
  }
  for (int l = 0; l < levels; ++l) {
    LevelCtx x{};
    x.sets = d_sets;
    x.act = d_act + P.act_off[l];
    x.act_next = l + 1 < levels ? d_act + P.act_off[l + 1] : nullptr;
    x.nact = (uint32_t)P.act[l].size();
    x.l = l;
    x.dim0 = P.dim0;
    x.rb = P.rb;
    x.err = err;
    x.local_next = P.use_local ? 1 : 0;
    x.vals_local = vals_local;
    const uint32_t n = P.items[l];
    // the buffer not holding vals_cur receives the level's first outputs
    uint32_t* vfree = vals_cur == valsA ? valsB : valsA;
    hcur = hist + P.hist_off[l];
    if (P.use_lists) {
      const int dl = (l + P.dim0) % k;  // the level's round-robin split dimension
      if (lazy && lat[dl] < l) KDB_CK(lift(dl, lat[dl], l, false));
      if (!(fold && l == 0)) KDB_CK(pivots_of(l));  // level 0's: taken while the lists were sorted
      // every list follows the level (sets leaving hand their lists over)
      if (!lazy)
        for (int d = 0; d < k; ++d) KDB_CK(lift(d, l, l + 1, false));
      if (tight && l + 1 < levels) {
        // split dimensions of level l + 1 from the first and last entries of
        // every subtree in each list
        TightArgs ta{};
        ta.x = x;
        for (int d = 0; d < k; ++d) ta.lists[d] = lcur[d];
        ta.items_next = P.items[l + 1];
        ta.dims = dims;
        ta.k = k;
        ta.ctype = P.ctype;
        Prof pf(K_WIDEST, (double)(x.nact << (l + 1)) * (2.0 * 16 * k + 1), 1, st);
        KDB_CK(launch_tight_children(ta, st));
      }
    } else if (P.seg[l]) {
      SegKeyArgs sa{};
      sa.x = x;
      sa.chunks = P.chunks[l];
      sa.vals = vals_cur;
      sa.vals_out = vfree;
      sa.ranks = ranks;
      sa.total = T;
      sa.k = k;
      sa.mode = P.mode;
      sa.dims = dims;
      sa.keys_out = reinterpret_cast<uint32_t*>(keysA);
      sa.seg_hist = hcur;
      sa.nseg = P.nseg[l];
      sa.passes = P.passes[l];
      {
        Prof pf(K_LEVEL_KEYS, (double)n * 12, 1, st);
        KDB_CK(launch_seg_level_keys(sa, st));
      }
      const uint32_t* kin = reinterpret_cast<uint32_t*>(keysA);
      const uint32_t* vin = vals_cur ? vals_cur : vfree;
      uint32_t* kout = reinterpret_cast<uint32_t*>(keysB);
      uint32_t* vout = vin == valsA ? valsB : valsA;
      for (int p = 0; p < P.passes[l]; ++p) {
        PassCtl c = ctl(n, 8 * p, nullptr);
        const uint32_t* sh = hcur + (size_t)p * P.nseg[l] * kRadixBins;
        if (p + 1 == P.passes[l]) {
          Prof pf(K_RADIX_UPDATE, (double)n * 12, 1, st);
          KDB_CK(seg_pass_update(kin, vin, x, sh, perm, vout, c, st));
          vals_cur = vout;
        } else {
          {
            Prof pf(K_RADIX, (double)n * 16, 1, st);
            KDB_CK(seg_pass_pingpong(kin, vin, kout, vout, x, sh, c, st));
          }
          const uint32_t* kt = kin;
          kin = kout;
          kout = const_cast<uint32_t*>(kt);
          const uint32_t* vt = vin;
          vin = vout;
          vout = const_cast<uint32_t*>(vt);
        }
      }
    } else {
    LevelKeyArgs ka{};
    ka.x = x;
    ka.items = n;
    ka.vals = vals_cur;
    ka.vals_out = vfree;  // level 0 only
    ka.ranks = ranks;
    ka.total = T;
    ka.k = k;
    ka.mode = P.mode;
    ka.dims = dims;
    ka.keys_out = keysA;
    ka.hist = hcur;
    ka.passes = P.passes[l];
    {
      Prof pf(K_LEVEL_KEYS, (double)n * 16, 1, st);
      KDB_CK(launch_level_keys(ka, sms, st));
    }
    const uint64_t* kin = keysA;
    const uint32_t* vin = vals_cur ? vals_cur : vfree;
    uint64_t* kout = keysB;
    uint32_t* vout = vin == valsA ? valsB : valsA;
    for (int p = 0; p < P.passes[l]; ++p) {
      PassCtl c = ctl(n, 8 * p, hcur + p * kRadixBins);
      if (p + 1 == P.passes[l]) {
        Prof pf(K_RADIX_UPDATE, (double)n * 16, 1, st);
        KDB_CK(pass_u64_update(kin, vin, x, perm, vout, c, st));
        vals_cur = vout;
      } else {
        {
          Prof pf(K_RADIX, (double)n * 24, 1, st);
          KDB_CK(pass_u64_pingpong(kin, vin, kout, vout, c, st));
        }
        const uint64_t* kt = kin;
        kin = kout;
        kout = const_cast<uint64_t*>(kt);
        const uint32_t* vt = vin;
        vin = vout;
        vout = const_cast<uint32_t*>(vt);
      }
    }
    }
    if (widest) {
      WidestArgs wa{};
      wa.x = x;
      wa.pts = pts;
      wa.k = k;
      wa.stride = P.stride;
      wa.perm = direct ? nullptr : perm;  // direct: the pivot's record is already at its node
      wa.boxes_in = (l & 1) ? boxB : boxA;
      wa.boxes_out = (l & 1) ? boxA : boxB;
      wa.dims = dims;
      wa.total_threads = x.nact << l;
      wa.boxes_local = boxes_local;
      wa.lsets = P.use_local ? d_lsets : nullptr;
      Prof pf(K_WIDEST, (double)(x.nact << l) * (2 * k * 4 * 3 + 8), 1, st);
      KDB_CK(launch_widest_children(wa, st));
    }
  }

  if (lazy && levels > 0) {
    // hand every list over to the local finish: the lists are independent,
    // so lists 1 .. k-1 go on side streams beside list 0, each with
    // look-back words of its own (not while `st` is being captured)
    const uint64_t words = ((uint64_t)std::max(T, P.max_items) + kPartTile - 1) / kPartTile * kLiftBins;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    KDB_CK(cudaStreamIsCapturing(st, &cap));
    const bool par = k > 1 && cap == cudaStreamCaptureStatusNone && (uint64_t)k * words <= (P.o_hist - P.o_status) / 8;
    if (!par) {
      for (int d = 0; d < k; ++d) KDB_CK(lift(d, lat[d], levels, true));
    } else {
      double bytes = 0.0;
      for (int d = 0; d < k; ++d) bytes += (double)P.items[lat[d]] * (16.0 + (lents && d == 0 ? 16.0 : 4.0));
      Prof phase(K_PARTITION, bytes, k, st, true, false);  // the lifts run side by side: timed as a whole
      SideStream side[2];
      for (int d = 1; d < k; ++d) {
        KDB_CK(side[d - 1].fork(st));
        KDB_CK(lift(d, lat[d], levels, true, side[d - 1].s, d * words, words, false));
        KDB_CK(side[d - 1].join(st));
      }
      KDB_CK(lift(0, lat[0], levels, true, st, 0, words, false));
      for (int d = 1; d < k; ++d) KDB_CK(side[d - 1].wait(st));
    }
  }

  // ---- subtrees small enough for one block: all remaining levels on chip
  if (P.use_local && !P.work.empty()) {
    LocalArgs la{};
    la.work = d_work;
    la.nwork = (uint32_t)P.work.size();
    la.lsets = d_lsets;
    la.vals_local = vals_local;
    la.lorig = P.use_lists ? lorig : nullptr;
    la.rows = P.use_lists ? ents0 : nullptr;
    la.ranks = P.use_lists ? nullptr : ranks;
    la.total = T;
    la.k = k;
    la.mode = P.mode;
    la.pts = pts;
    la.stride = P.stride;
    la.boxes_local = boxes_local;
    la.bbox = bbox;
    la.dims = dims;
    la.perm = perm;
    la.err = err;
    la.lents = lents;
    la.pts_out = direct ? pts : nullptr;
    la.ctype = P.ctype;
    la.dim0 = P.dim0;
    // algorithmic bytes per point: the handed-over lists in (list 0 as
    // entries when handed over whole), perm out, and the record written at
    // its node when it is written from its entry
    const double lin = P.use_lists ? (lents ? 16.0 + 4.0 * (k - 1) : 4.0 * k) : 4.0 + 4.0 * k;
    Prof pf(K_LOCAL, (double)T * (lin + 4.0 + (direct ? (double)P.stride : 0.0)), 1, st);
    KDB_CK(launch_local_finish(la, st));
  }

  // ---- placement
  if (out_dim && !bydim) {
    Prof pf(K_WIDEST, (double)T, 1, st);
    KDB_CK(launch_rr_dims(dims, d_sets, (uint32_t)P.sets.size(), T, k, P.dim0, st));
  }
  PermuteArgs pm{};
  pm.pts = pts;
  pm.total = T;
  pm.stride = P.stride;
  pm.perm = perm;
  pm.stage = at<unsigned char>(ws, P.o_stage);
  pm.err = err;
  if (direct) {
    // every record is at its node already; put the input back if the build failed
    Prof pf(K_PLACEMENT, 0.0, 1, st);
    KDB_CK(launch_restore(pts, ents0, T, k, err, P.ctype, st));
  } else if (placement == KDB_PLACEMENT_AUTO && (size_t)T * P.stride <= P.gather_bytes) {
    Prof pf(K_PLACEMENT, (double)T * (4.0 + 4.0 * P.stride), 2, st);
    KDB_CK(launch_place_gather(pm, at<unsigned char>(ws, P.o_gather), sms, st));
  } else {
    Prof pf(K_PLACEMENT, (double)T * (4.0 + 2.0 * P.stride), 5, st);
    KDB_CK(launch_permute(pm, sms, st));
  }
  if (out_orig) {
    Prof pf(K_PLACEMENT, (double)T * 8, 1, st);
    KDB_CK(launch_unmark(perm, out_orig, T, st));
  }
  if (out_dim) KDB_CK(cudaMemcpyAsync(out_dim, dims, T, cudaMemcpyDeviceToDevice, st));
  return KDB_OK;
}

kdb_status finish(const Plan& P, void* ws, cudaStream_t st) {
  uint32_t h_err = 0;
  KDB_CK(cudaMemcpyAsync(&h_err, at<uint32_t>(ws, P.o_err), 4, cudaMemcpyDeviceToHost, st));
  KDB_CK(cudaStreamSynchronize(st));
  if (h_err & ERR_NAN) return KDB_ERR_NAN_INPUT;
  if (h_err & ERR_TIMEOUT) return KDB_ERR_TIMEOUT;
  if (h_err & ERR_INTERNAL) return KDB_ERR_INTERNAL;
  return KDB_OK;
}

kdb_status run(Plan& P, unsigned char* pts, void* user_ws, size_t user_bytes, int32_t* out_orig,
               uint8_t* out_dim, cudaStream_t st, bool planned = false) {
  if (!planned) make_plan(P);
  if (P.too_wide) return KDB_ERR_INVALID_ARGUMENT;
  int dev, sms;
  cudaMemPool_t pool;
  kdb_status s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  void* ws = user_ws;
  if (ws) {
    if (user_bytes < P.bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return KDB_ERR_INVALID_ARGUMENT;
  } else {
    s = pool_alloc(&ws, P.bytes, pool, st);
    if (s != KDB_OK) return s;
  }
  s = enqueue_build(P, pts, ws, sms, out_orig, out_dim, st);
  kdb_status f = finish(P, ws, st);
  if (!user_ws) {
    cudaFreeAsync(ws, st);
    cudaStreamSynchronize(st);
  }
  return s != KDB_OK ? s : f;
}

// run() for a cached plan: the tables come from its pinned image.
kdb_status run_cached(const CachedPlan& C, unsigned char* pts, void* user_ws, size_t user_bytes,
                      int32_t* out_orig, uint8_t* out_dim, cudaStream_t st) {
  const Plan& P = C.P;
  if (P.too_wide) return KDB_ERR_INVALID_ARGUMENT;
  int dev, sms;
  cudaMemPool_t pool;
  kdb_status s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  void* ws = user_ws;
  if (ws) {
    if (user_bytes < P.bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return KDB_ERR_INVALID_ARGUMENT;
  } else {
    s = pool_alloc(&ws, P.bytes, pool, st);
    if (s != KDB_OK) return s;
  }
  bool ready = false;
  if (C.h_img) {
    if (cudaMemcpyAsync(static_cast<unsigned char*>(ws) + C.img_off, C.h_img, C.img_bytes,
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      s = KDB_ERR_CUDA;
    }
    ready = true;
  }
  if (s == KDB_OK) s = enqueue_build(P, pts, ws, sms, out_orig, out_dim, st, ready);
  kdb_status f = finish(P, ws, st);
  if (!user_ws) {
    cudaFreeAsync(ws, st);
    cudaStreamSynchronize(st);
  }
  return s != KDB_OK ? s : f;
}

// ------------------------------------------------------- no-alloc build --
// Workspace of kdb_build_noalloc: one static device array per GPU that loads
// the library.  Host code must not use the symbol's host-side address; the
// device address is looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KDB_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

kdb_status noalloc_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return KDB_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return KDB_OK;
}

}  // namespace

// A build prepared once and enqueued many times (kdb_plan_*).
struct PlanObj {
  Plan P;
  void* ws = nullptr;
  int dev = 0, sms = 1;
  uint32_t* h_err = nullptr;  // pinned
  bool trivial = false;       // N <= 1 in every set: nothing to do
};

cudaError_t ensure_smem(const void* func, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (SmemAttr& a : g_attr) {
    if (a.dev != dev || a.func != func) continue;
    if (a.bytes >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) a.bytes = bytes;
    return e;
  }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) g_attr.push_back({dev, func, bytes});
  return e;
}
}  // namespace kdb

// ------------------------------------------------------ memory-lean build --
// A single build in a small workspace, on one GPU, by the steps of the
// sharded build with every shard on this GPU: the top g levels are chosen
// over the whole array (per node the point of rank ss(lChild) in the node's
// order, Observation 1, by a radix select over (coordinate key << 32 |
// index)), every point is moved once to its level-g subtree's slice (a
// stable partition), and each of the 2^g subtrees is then built alone with
// the ordinary pipeline in a workspace sized for one subtree.  The caller's
// records are only read until every subtree is built; the tree is written
// into them at the end.
namespace kdb {
namespace {
std::atomic<int> g_memory_mode{KDB_MEMORY_AUTO};
constexpr int kLeanLevels = 4;  // 16 subtrees: each build's workspace is about 1/16 of one over all points
constexpr uint32_t kLeanCand = 4096;  // points of one coordinate key gathered per node, at most

// Widest side of a box of coordinate keys, as the device's widest_of_keys:
// float32 hi - lo (exact key differences for integer coordinates), strict
// '>' from d = 0, so the lowest dimension wins ties.
int host_widest(const uint32_t* lo, const uint32_t* hi, int k, int ctype) {
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
    const uint32_t hb = key_to_float_bits(hi[d]), lb = key_to_float_bits(lo[d]);
    float hf, lf;
    std::memcpy(&hf, &hb, 4);
    std::memcpy(&lf, &lb, 4);
    const float e = hf - lf;
    if (d == 0 || e > be) {
      be = e;
      best = d;
    }
  }
  return best;
}

struct LeanPlan {
  int g = 0;                 // levels chosen over the whole array
  uint32_t G = 0;            // subtrees
  std::vector<uint32_t> m;   // points of each subtree
  size_t sub_bytes = 0;      // workspace of the largest subtree build
  uint32_t blocks = 0;       // partition blocks
  size_t o_tags, o_out, o_idx, o_hist, o_box, o_dims, o_pre, o_pin, o_top, o_cnt, o_cand, o_err, o_ws, bytes;
};

// Layout of the lean build's device memory; g = 0 if n is too small for it.
LeanPlan lean_plan(int64_t n, int k, int stride, int mode_arg, int sms) {
  LeanPlan L;
  const uint32_t N = (uint32_t)n;
  L.g = std::min(kLeanLevels, num_levels(N) - 2);  // levels 0..g full
  if (L.g < 1) {
    L.g = 0;
    return L;
  }
  L.G = 1u << L.g;
  const Tree t = make_tree(N);
  for (uint32_t r = 0; r < L.G; ++r) {
    L.m.push_back(subtree_size(t, full_nodes(L.g) + r));
    Plan P;
    P.sets.push_back(SetInfo{0u, L.m.back()});
    P.total = L.m.back();
    P.k = k;
    P.stride = stride;
    P.mode = mode_arg & 0xFF;
    P.ctype = ctype_of(mode_arg);
    P.mode_arg = mode_arg;
    make_plan(P);
    L.sub_bytes = std::max(L.sub_bytes, P.bytes);
  }
  L.blocks = dist_blocks(N, sms);
  const uint32_t top_nodes = 1u << (L.g - 1);  // most nodes of a chosen level
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  L.o_tags = take((size_t)N * 4);
  L.o_out = take((size_t)N * stride);
  L.o_idx = take((size_t)N * 4);
  L.o_hist = take((size_t)top_nodes * 256 * 4);
  L.o_box = take((size_t)top_nodes * 2 * k * 4);
  L.o_dims = take(top_nodes);
  L.o_pre = take((size_t)top_nodes * 8);
  L.o_pin = take((size_t)top_nodes * 8);
  L.o_top = take((size_t)full_nodes(L.g) * stride);
  L.o_cnt = take((size_t)L.blocks * L.G * 8);
  L.o_cand = take((size_t)top_nodes * (kLeanCand + 1) * 4);
  L.o_err = take(4);
  L.o_ws = take(L.sub_bytes);
  L.bytes = off;
  return L;
}

kdb_status lean_build(unsigned char* pts, int64_t n, int k, int stride, int mode_arg, cudaStream_t st) {
  int dev, sms;
  cudaMemPool_t pool;
  kdb_status s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  const LeanPlan L = lean_plan(n, k, stride, mode_arg, sms);
  if (L.g == 0) return KDB_ERR_INVALID_ARGUMENT;
  const uint32_t N = (uint32_t)n;
  const int split = mode_arg & 0xFF, ctype = ctype_of(mode_arg);
  const Tree tree = make_tree(N);
  void* ws = nullptr;
  s = pool_alloc(&ws, L.bytes, pool, st);
  if (s != KDB_OK) return s;
  unsigned char* base = static_cast<unsigned char*>(ws);
  int32_t* tags = reinterpret_cast<int32_t*>(base + L.o_tags);
  unsigned char* out = base + L.o_out;
  uint32_t* idx = reinterpret_cast<uint32_t*>(base + L.o_idx);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + L.o_hist);
  uint32_t* box = reinterpret_cast<uint32_t*>(base + L.o_box);
  uint8_t* d_dims = base + L.o_dims;
  uint64_t* d_pre = reinterpret_cast<uint64_t*>(base + L.o_pre);
  int64_t* d_pin = reinterpret_cast<int64_t*>(base + L.o_pin);
  unsigned char* top = base + L.o_top;
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + L.o_cnt);
  uint32_t* cand = reinterpret_cast<uint32_t*>(base + L.o_cand);  // [nodes] counts, then [nodes][kLeanCand]
  uint32_t* err = reinterpret_cast<uint32_t*>(base + L.o_err);
  void* sub_ws = base + L.o_ws;
  kdb_status result = KDB_OK;
  // a device error word read back after each host decision
  auto sync_err = [&](uint32_t* h) -> kdb_status {
    uint32_t e = 0;
    if (cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return KDB_ERR_CUDA;
    if (h) *h = e;
    if (e & ERR_NAN) return KDB_ERR_NAN_INPUT;
    if (e & ERR_TIMEOUT) return KDB_ERR_TIMEOUT;
    if (e & ERR_INTERNAL) return KDB_ERR_INTERNAL;
    return KDB_OK;
  };
  DistArgs a{};
  a.pts = pts;
  a.n = N;
  a.k = k;
  a.stride = stride;
  a.ctype = ctype;
  a.tags = tags;
  a.err = err;
  do {
    if (cudaMemsetAsync(err, 0, 4, st) != cudaSuccess || cudaMemsetAsync(tags, 0, (size_t)N * 4, st) != cudaSuccess) {
      result = KDB_ERR_CUDA;
      break;
    }
    if (ctype == kCoordF32) {  // NaN coordinates: refused before anything is built
      Prof pf(K_LEAN, (double)N * 4 * k, 1, st);
      if (launch_nan_check(pts, N, k, stride, err, sms, st) != cudaSuccess) {
        result = KDB_ERR_CUDA;
        break;
      }
    }
    if ((result = sync_err(nullptr)) != KDB_OK) break;
    // top levels: per level the split dimensions, a radix select of every
    // node's pivot and the tag update
    std::vector<uint32_t> dom_lo, dom_hi;  // widest extent: node domains as keys, heap order
    auto read_boxes = [&](int l, std::vector<uint32_t>* h) -> kdb_status {
      a.first = full_nodes(l);
      a.nodes = 1u << l;
      a.box = box;
      std::vector<uint32_t> init((size_t)a.nodes * 2 * k);
      for (size_t i = 0; i < init.size(); ++i) init[i] = (i / k) % 2 == 0 ? 0xFFFFFFFFu : 0u;
      h->resize(init.size());
      Prof pf(K_LEAN, (double)N * (4.0 * k + 4.0), 1, st);
      if (cudaMemcpyAsync(box, init.data(), init.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          launch_dist_box(a, sms, st) != cudaSuccess ||
          cudaMemcpyAsync(h->data(), box, init.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return KDB_ERR_CUDA;
      return sync_err(nullptr);
    };
    if (split == KDB_SPLIT_WIDEST_EXTENT) {
      std::vector<uint32_t> b;
      if ((result = read_boxes(0, &b)) != KDB_OK) break;
      dom_lo.assign((size_t)full_nodes(L.g + 1) * k, 0);
      dom_hi.assign((size_t)full_nodes(L.g + 1) * k, 0);
      for (int d = 0; d < k; ++d) {
        dom_lo[d] = b[d];
        dom_hi[d] = b[k + d];
      }
    }
    for (int l = 0; l < L.g && result == KDB_OK; ++l) {
      const uint32_t nodes = 1u << l, first = full_nodes(l);
      std::vector<uint8_t> dims(nodes);
      if (split == KDB_SPLIT_ROUND_ROBIN) {
        for (uint32_t u = 0; u < nodes; ++u) dims[u] = (uint8_t)(l % k);
      } else if (split == KDB_SPLIT_WIDEST_EXTENT) {
        for (uint32_t u = 0; u < nodes; ++u)
          dims[u] = (uint8_t)host_widest(&dom_lo[(size_t)(first + u) * k], &dom_hi[(size_t)(first + u) * k], k, ctype);
      } else {
        std::vector<uint32_t> b;
        if ((result = read_boxes(l, &b)) != KDB_OK) break;
        for (uint32_t u = 0; u < nodes; ++u)
          dims[u] = (uint8_t)host_widest(&b[(size_t)u * 2 * k], &b[(size_t)u * 2 * k + k], k, ctype);
      }
      std::vector<uint64_t> remaining(nodes), prefix(nodes, 0);
      for (uint32_t u = 0; u < nodes; ++u) remaining[u] = subtree_size(tree, 2 * (first + u) + 1);
      a.first = first;
      a.nodes = nodes;
      a.node_dim = d_dims;
      a.prefix = d_pre;
      a.hist = hist;
      if (cudaMemcpyAsync(d_dims, dims.data(), nodes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        result = KDB_ERR_CUDA;
        break;
      }
      std::vector<uint32_t> h((size_t)nodes * 256);
      for (int rnd = 0; rnd < 8 && result == KDB_OK; ++rnd) {
        if (rnd == 4) {
          // the coordinate keys are fixed: gather every node's points with
          // its key; the pivot is the one of rank remaining[u] among them by
          // index (four histogram passes over all points otherwise)
          std::vector<uint32_t> cc(nodes), cl((size_t)nodes * kLeanCand);
          Prof pf(K_LEAN, (double)N * 8.0, 1, st);
          if (cudaMemcpyAsync(d_pre, prefix.data(), (size_t)nodes * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemsetAsync(cand, 0, (size_t)nodes * 4, st) != cudaSuccess ||
              launch_lean_collect(a, kLeanCand, cand, cand + nodes, sms, st) != cudaSuccess ||
              cudaMemcpyAsync(cc.data(), cand, (size_t)nodes * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaMemcpyAsync(cl.data(), cand + nodes, cl.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            result = KDB_ERR_CUDA;
            break;
          }
          if ((result = sync_err(nullptr)) != KDB_OK) break;
          bool all = true;
          for (uint32_t u = 0; u < nodes; ++u) all = all && cc[u] <= kLeanCand && remaining[u] < cc[u];
          if (all) {
            for (uint32_t u = 0; u < nodes; ++u) {
              uint32_t* c0 = cl.data() + (size_t)u * kLeanCand;
              std::nth_element(c0, c0 + remaining[u], c0 + cc[u]);
              prefix[u] = (prefix[u] << 32) | c0[remaining[u]];
            }
            break;  // every pivot is known
          }
        }
        a.prefix_bits = 8 * rnd;
        Prof pf(K_LEAN, (double)N * 8.0, 1, st);
        if (cudaMemcpyAsync(d_pre, prefix.data(), (size_t)nodes * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(hist, 0, h.size() * 4, st) != cudaSuccess || launch_dist_hist(a, sms, st) != cudaSuccess ||
            cudaMemcpyAsync(h.data(), hist, h.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
          result = KDB_ERR_CUDA;
          break;
        }
        if ((result = sync_err(nullptr)) != KDB_OK) break;
        for (uint32_t u = 0; u < nodes; ++u) {
          // the digit of the pivot: the bucket holding rank remaining[u]
          uint64_t cum = 0;
          int dgt = 0;
          while (dgt < 256 && cum + h[(size_t)u * 256 + dgt] <= remaining[u]) cum += h[(size_t)u * 256 + dgt++];
          if (dgt == 256) {
            result = KDB_ERR_INTERNAL;
            break;
          }
          remaining[u] -= cum;
          prefix[u] = (prefix[u] << 8) | (uint64_t)dgt;
        }
      }
      if (result != KDB_OK) break;
      std::vector<int64_t> pinned(nodes, -1);
      a.pivot = d_pre;
      a.pinned = d_pin;
      {
        Prof pf(K_LEAN, (double)N * 12.0, 1, st);
        if (cudaMemcpyAsync(d_pre, prefix.data(), (size_t)nodes * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(d_pin, 0xFF, (size_t)nodes * 8, st) != cudaSuccess ||
            launch_dist_assign(a, sms, st) != cudaSuccess ||
            cudaMemcpyAsync(pinned.data(), d_pin, (size_t)nodes * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
          result = KDB_ERR_CUDA;
          break;
        }
      }
      if ((result = sync_err(nullptr)) != KDB_OK) break;
      for (uint32_t u = 0; u < nodes && result == KDB_OK; ++u) {
        if (pinned[u] < 0 || pinned[u] >= (int64_t)N || (uint64_t)pinned[u] != (prefix[u] & 0xFFFFFFFFu)) {
          result = KDB_ERR_INTERNAL;
          break;
        }
        // the pivot's record, kept for its node
        if (cudaMemcpyAsync(top + (size_t)(first + u) * stride, pts + (size_t)pinned[u] * stride, stride,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          result = KDB_ERR_CUDA;
        if (split == KDB_SPLIT_WIDEST_EXTENT) {  // the children's domains, clipped at the pivot's plane
          const uint32_t plane = (uint32_t)(prefix[u] >> 32);
          const size_t s0 = (size_t)(first + u) * k, lc = (size_t)(2 * (first + u) + 1) * k, rc = lc + k;
          for (int d = 0; d < k; ++d) {
            dom_lo[lc + d] = dom_lo[rc + d] = dom_lo[s0 + d];
            dom_hi[lc + d] = dom_hi[rc + d] = dom_hi[s0 + d];
          }
          dom_hi[lc + dims[u]] = plane;
          dom_lo[rc + dims[u]] = plane;
        }
      }
    }
    if (result != KDB_OK) break;
    // every point to its level-g subtree's slice, in original-index order
    a.first = full_nodes(L.g);
    a.nodes = L.G;
    a.out_pts = out;
    a.out_index = idx;
    a.block_counts = cnt;
    const size_t cells = (size_t)L.blocks * L.G;
    std::vector<uint32_t> bc(cells), off(cells);
    {
      Prof pf(K_LEAN, (double)N * 4.0, 1, st);
      if (launch_dist_count(a, L.blocks, st) != cudaSuccess ||
          cudaMemcpyAsync(bc.data(), cnt, cells * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        result = KDB_ERR_CUDA;
        break;
      }
    }
    std::vector<uint32_t> start(L.G + 1, 0);
    uint64_t run = 0;
    for (uint32_t r = 0; r < L.G; ++r) {
      start[r] = (uint32_t)run;
      for (uint32_t b = 0; b < L.blocks; ++b) {
        off[(size_t)b * L.G + r] = (uint32_t)run;
        run += bc[(size_t)b * L.G + r];
      }
      if (run - start[r] != L.m[r]) result = KDB_ERR_INTERNAL;  // the subtree's size is fixed by N
    }
    start[L.G] = (uint32_t)run;
    if (result != KDB_OK) break;
    a.block_offsets = cnt + cells;
    {
      Prof pf(K_LEAN, (double)N * (2.0 * stride + 8.0), 1, st);
      if (cudaMemcpyAsync(cnt + cells, off.data(), cells * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          launch_dist_scatter(a, L.blocks, st) != cudaSuccess) {
        result = KDB_ERR_CUDA;
        break;
      }
    }
    if ((result = sync_err(nullptr)) != KDB_OK) break;
    // each subtree alone: round robin continued from its level, or its
    // domain clipped by its ancestors' planes
    for (uint32_t r = 0; r < L.G && result == KDB_OK; ++r) {
      Plan P;
      P.sets.push_back(SetInfo{0u, L.m[r]});
      P.total = L.m[r];
      P.k = k;
      P.stride = stride;
      P.mode = split;
      P.ctype = ctype;
      P.mode_arg = mode_arg;
      P.dim0 = split == KDB_SPLIT_ROUND_ROBIN ? L.g % k : 0;
      if (split == KDB_SPLIT_WIDEST_EXTENT) {
        P.has_domain = true;
        const size_t s0 = (size_t)(full_nodes(L.g) + r) * k;
        for (int d = 0; d < k; ++d) {
          const uint32_t lb = key_to_float_bits(dom_lo[s0 + d]), hb = key_to_float_bits(dom_hi[s0 + d]);
          std::memcpy(&P.domain[d], &lb, 4);
          std::memcpy(&P.domain[kMaxK + d], &hb, 4);
        }
      }
      make_plan(P);
      if (P.too_wide || P.bytes > L.sub_bytes) {
        result = KDB_ERR_INTERNAL;
        break;
      }
      if (L.m[r] <= 1) continue;
      result = enqueue_build(P, out + (size_t)start[r] * stride, sub_ws, sms, nullptr, nullptr, st);
      const kdb_status f = finish(P, sub_ws, st);
      if (result == KDB_OK) result = f;
    }
    if (result != KDB_OK) break;
    // every subtree and the top nodes into the caller's array
    for (uint32_t r = 0; r < L.G && result == KDB_OK; ++r) {
      LeanPlaceArgs pa{};
      pa.src = out + (size_t)start[r] * stride;
      pa.dst = pts;
      pa.m = L.m[r];
      pa.total = N;
      pa.g = L.g;
      pa.rank = r;
      pa.stride = stride;
      pa.err = err;
      Prof pf(K_PLACEMENT, (double)L.m[r] * 2.0 * stride, 1, st);
      if (launch_lean_place(pa, st) != cudaSuccess) result = KDB_ERR_CUDA;
    }
    if (result != KDB_OK) break;
    if (cudaMemcpyAsync(pts, top, (size_t)full_nodes(L.g) * stride, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      result = KDB_ERR_CUDA;
      break;
    }
    result = sync_err(nullptr);
  } while (0);
  if (result == KDB_ERR_CUDA) cudaGetLastError();
  cudaFreeAsync(ws, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && result == KDB_OK) result = KDB_ERR_CUDA;
  return result;
}

// Whether an automatic build goes the lean way: its ordinary workspace does
// not fit the device memory free now (free memory plus what the library's
// pool holds unused), less a margin.
bool lean_needed(size_t ws_bytes) {
  if (g_fault == KDB_FAULT_LOW_MEMORY) {  // tests: as if only g_fault_arg bytes were free
    g_fault = KDB_FAULT_NONE;
    return ws_bytes + ((size_t)256 << 20) > (size_t)std::max<int64_t>(g_fault_arg, 0);
  }
  int dev, sms;
  cudaMemPool_t pool;
  if (device_setup(&dev, &pool, &sms) != KDB_OK) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  uint64_t reserved = 0, used = 0;
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  const size_t avail = free_b + (size_t)(reserved > used ? reserved - used : 0);
  const size_t margin = (size_t)256 << 20;
  return ws_bytes + margin > avail;
}
}  // namespace
}  // namespace kdb


using namespace kdb;

extern "C" {

const char* kdb_status_string(kdb_status s) {
  switch (s) {
    case KDB_OK: return "ok";
    case KDB_ERR_INVALID_ARGUMENT: return "invalid argument";
    case KDB_ERR_OUT_OF_MEMORY: return "out of device memory";
    case KDB_ERR_CUDA: return "CUDA error";
    case KDB_ERR_NAN_INPUT: return "NaN coordinate in input";
    case KDB_ERR_TIMEOUT: return "bounded device wait timed out";
    case KDB_ERR_NOT_A_KD_TREE: return "not a k-d tree";
    case KDB_ERR_INTERNAL: return "internal consistency check failed";
  }
  return "unknown status";
}

int kdb_version(void) { return 100; }

void kdb_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = true;
}

int kdb_profile_stop(kdb_kernel_stat* out, int max_entries) {
  std::vector<ProfRec> recs;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    recs.swap(g_prof);
  }
  kdb_kernel_stat agg[K_COUNT];
  memset(agg, 0, sizeof agg);
  bool ok = true;
  for (const ProfRec& r : recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
    agg[r.kind].launches += r.launches;
    agg[r.kind].ms += ms;
    agg[r.kind].bytes += r.bytes;
  }
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const ProfRec& r : recs) {
      g_event_pool.push_back(r.a);
      g_event_pool.push_back(r.b);
    }
  }
  if (!ok) return -1;
  int n = 0;
  for (int kd = 0; kd < K_COUNT; ++kd) {
    if (!agg[kd].launches) continue;
    if (out && n < max_entries) {
      out[n] = agg[kd];
      snprintf(out[n].name, sizeof out[n].name, "%s", kKindName[kd]);
    }
    ++n;
  }
  return n < max_entries ? n : max_entries;
}

int64_t kdb_launch_count(void) { return g_launches.load(); }

kdb_placement kdb_set_placement(kdb_placement placement) {
  if (placement != KDB_PLACEMENT_AUTO && placement != KDB_PLACEMENT_IN_PLACE)
    return (kdb_placement)g_placement.load();
  return (kdb_placement)g_placement.exchange(placement);
}

int kdb_tuning_shape_count(int kernel) {
  if (kernel == KDB_TUNE_PARTITION) return kPartShapes;
  if (kernel == KDB_TUNE_RADIX) return kRecShapes;
  if (kernel == KDB_TUNE_DIGITS) return kRecDigitWidths;
  return -1;
}

kdb_status kdb_tuning_shape(int kernel, int index, int* threads, int* items_per_thread,
                            int* blocks_per_sm) {
  const int count = kdb_tuning_shape_count(kernel);
  if (count < 0 || index < 0 || index >= count) return KDB_ERR_INVALID_ARGUMENT;
  if (kernel == KDB_TUNE_DIGITS) {  // width in bits, passes per 32-bit key
    if (threads) *threads = kRecDigitBits[index];
    if (items_per_thread) *items_per_thread = rec_passes(kRecDigitBits[index]);
    if (blocks_per_sm) *blocks_per_sm = 1;
    return KDB_OK;
  }
  const TileShape& sh = kernel == KDB_TUNE_PARTITION ? kPartShape[index] : kRecShape[index];
  if (threads) *threads = sh.threads;
  if (items_per_thread) *items_per_thread = sh.items;
  if (blocks_per_sm) *blocks_per_sm = sh.blocks;
  return KDB_OK;
}

namespace {
int width_index(int bits) {
  for (int i = 0; i < kRecDigitWidths; ++i)
    if (kRecDigitBits[i] == bits) return i;
  return -1;
}
bool tuning_valid(const kdb_tuning& t) {
  return t.partition_shape >= 0 && t.partition_shape < kPartShapes && t.radix_shape >= 0 &&
         t.radix_shape < kRecShapes && width_index(t.digit_bits) >= 0;
}
}  // namespace

kdb_status kdb_get_tuning(kdb_tuning* out) {
  if (!out) return KDB_ERR_INVALID_ARGUMENT;
  out->partition_shape = g_part_shape.load();
  out->radix_shape = g_rec_shape.load();
  out->digit_bits = g_rec_bits.load();
  return KDB_OK;
}

kdb_status kdb_set_tuning(const kdb_tuning* t) {
  if (!t || !tuning_valid(*t)) return KDB_ERR_INVALID_ARGUMENT;
  g_part_shape.store(t->partition_shape);
  g_rec_shape.store(t->radix_shape);
  g_rec_bits.store(t->digit_bits);
  return KDB_OK;
}

kdb_status kdb_lookup_tuning(int64_t n, int k, int stride_bytes, kdb_split_mode mode, kdb_tuning* out,
                             int* from_table) {
  if (!out || n < 0) return KDB_ERR_INVALID_ARGUMENT;
  bool found = false;
  const TuneEntry e = tuning_for((uint64_t)n, k, stride_bytes, (int)mode, &found);
  *out = kdb_tuning{e.part, e.rec, e.bits};
  if (from_table) *from_table = found ? 1 : 0;
  return KDB_OK;
}

void kdb_clear_tuning_table(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_table.clear();
}

kdb_status kdb_save_tuning(const char* path) {
  if (!path) return KDB_ERR_INVALID_ARGUMENT;
  std::vector<TuneEntry> table;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    table = g_tune_table;
  }
  FILE* f = fopen(path, "w");
  if (!f) return KDB_ERR_INVALID_ARGUMENT;
  auto shape = [](const TileShape& sh) {
    char b[64];
    snprintf(b, sizeof b, "[%d, %d, %d]", sh.threads, sh.items, sh.blocks);
    return std::string(b);
  };
  std::string text = "{\"partition\": " + shape(kPartShape[g_part_shape.load()]) +
                     ", \"radix\": " + shape(kRecShape[g_rec_shape.load()]) +
                     ", \"digit_bits\": " + std::to_string(g_rec_bits.load()) + ", \"table\": [";
  for (size_t i = 0; i < table.size(); ++i) {
    const TuneEntry& e = table[i];
    text += (i ? ",\n  " : "\n  ");
    text += "{\"log2n\": " + std::to_string(e.log2n) + ", \"k\": " + std::to_string(e.k) +
            ", \"stride\": " + std::to_string(e.stride) + ", \"mode\": " + std::to_string(e.mode) +
            ", \"partition\": " + shape(kPartShape[e.part]) + ", \"radix\": " + shape(kRecShape[e.rec]) +
            ", \"digit_bits\": " + std::to_string(e.bits) + "}";
  }
  text += "]}\n";
  const size_t w = fwrite(text.data(), 1, text.size(), f);
  return (fclose(f) == 0 && w == text.size()) ? KDB_OK : KDB_ERR_INVALID_ARGUMENT;
}

namespace {
// A small JSON reader for the tuning file: objects, arrays, integers and
// plain strings (no escapes), nested at most four deep.
struct JVal {
  enum Kind { NONE, INT, STR, ARR, OBJ } kind = NONE;
  long long num = 0;
  std::string str;
  std::vector<std::string> keys;  // OBJ: parallel to items
  std::vector<JVal> items;        // ARR elements or OBJ values
  const JVal* get(const char* key) const {
    if (kind != OBJ) return nullptr;
    for (size_t i = 0; i < keys.size(); ++i)
      if (keys[i] == key) return &items[i];
    return nullptr;
  }
};

struct JReader {
  const char* p;
  const char* end;
  void ws() {
    while (p < end && (*p == ' ' || *p == '\t' || *p == '\r' || *p == '\n')) ++p;
  }
  bool text(std::string& s) {
    if (p >= end || *p != '"') return false;
    const char* b = ++p;
    while (p < end && *p != '"') {
      if (*p == '\\' || (unsigned char)*p < 0x20) return false;
      ++p;
    }
    if (p >= end || p - b > 64) return false;
    s.assign(b, p);
    ++p;
    return true;
  }
  bool value(JVal& v, int depth) {
    if (depth > 4) return false;
    ws();
    if (p >= end) return false;
    if (*p == '{' || *p == '[') {
      const bool obj = *p == '{';
      const char close = obj ? '}' : ']';
      v.kind = obj ? JVal::OBJ : JVal::ARR;
      ++p;
      ws();
      if (p < end && *p == close) {
        ++p;
        return true;
      }
      for (;;) {
        if (v.items.size() >= 4096) return false;
        if (obj) {
          ws();
          std::string key;
          if (!text(key)) return false;
          ws();
          if (p >= end || *p != ':') return false;
          ++p;
          v.keys.push_back(key);
        }
        v.items.emplace_back();
        if (!value(v.items.back(), depth + 1)) return false;
        ws();
        if (p >= end) return false;
        if (*p == ',') {
          ++p;
          continue;
        }
        if (*p != close) return false;
        ++p;
        return true;
      }
    }
    if (*p == '"') {
      v.kind = JVal::STR;
      return text(v.str);
    }
    const bool neg = *p == '-';
    if (neg) ++p;
    long long x = 0;
    int digits = 0;
    while (p < end && *p >= '0' && *p <= '9') {
      if (++digits > 12) return false;
      x = 10 * x + (*p - '0');
      ++p;
    }
    if (digits == 0) return false;
    v.kind = JVal::INT;
    v.num = neg ? -x : x;
    return true;
  }
};

bool json_int(const JVal* v, long long lo, long long hi, int* out) {
  if (!v || v->kind != JVal::INT || v->num < lo || v->num > hi) return false;
  *out = (int)v->num;
  return true;
}

// index of the compiled shape stored by value as [threads, items, blocks]
int json_shape(const JVal* v, const TileShape* table, int count) {
  if (!v || v->kind != JVal::ARR || v->items.size() != 3) return -1;
  int x[3];
  for (int i = 0; i < 3; ++i)
    if (!json_int(&v->items[i], 1, 4096, &x[i])) return -1;
  for (int i = 0; i < count; ++i)
    if (table[i].threads == x[0] && table[i].items == x[1] && table[i].blocks == x[2]) return i;
  return -1;
}

// a setting: "partition", "radix" and (default 8) "digit_bits"
bool json_tuning(const JVal& o, kdb_tuning* t) {
  t->partition_shape = json_shape(o.get("partition"), kPartShape, kPartShapes);
  t->radix_shape = json_shape(o.get("radix"), kRecShape, kRecShapes);
  t->digit_bits = 8;
  const JVal* b = o.get("digit_bits");
  if (b && !json_int(b, 1, 32, &t->digit_bits)) return false;
  return tuning_valid(*t);
}
}  // namespace

kdb_status kdb_load_tuning(const char* path) {
  if (!path) return KDB_ERR_INVALID_ARGUMENT;
  FILE* f = fopen(path, "r");
  if (!f) return KDB_ERR_INVALID_ARGUMENT;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof buf, f)) > 0 && text.size() <= (1u << 18)) text.append(buf, got);
  fclose(f);
  if (text.size() > (1u << 18)) return KDB_ERR_INVALID_ARGUMENT;
  JVal root;
  JReader r{text.data(), text.data() + text.size()};
  if (!r.value(root, 0) || root.kind != JVal::OBJ) return KDB_ERR_INVALID_ARGUMENT;
  r.ws();
  if (r.p != r.end) return KDB_ERR_INVALID_ARGUMENT;
  kdb_tuning g{};
  if (!json_tuning(root, &g)) return KDB_ERR_INVALID_ARGUMENT;
  std::vector<TuneEntry> table;
  if (const JVal* tv = root.get("table")) {  // absent: an empty table
    if (tv->kind != JVal::ARR || tv->items.size() > (size_t)kTuneTableMax) return KDB_ERR_INVALID_ARGUMENT;
    for (const JVal& o : tv->items) {
      if (o.kind != JVal::OBJ) return KDB_ERR_INVALID_ARGUMENT;
      TuneEntry e{};
      kdb_tuning t{};
      if (!json_int(o.get("log2n"), 0, 64, &e.log2n) || !json_int(o.get("k"), 1, kMaxK, &e.k) ||
          !json_int(o.get("stride"), 1, 1 << 24, &e.stride) || !json_int(o.get("mode"), 0, 1 << 16, &e.mode) ||
          !json_tuning(o, &t))
        return KDB_ERR_INVALID_ARGUMENT;
      e.part = t.partition_shape;
      e.rec = t.radix_shape;
      e.bits = t.digit_bits;
      bool dup = false;  // a repeated kind: the later entry wins
      for (TuneEntry& x : table)
        if (x.log2n == e.log2n && x.k == e.k && x.stride == e.stride && x.mode == e.mode) {
          x = e;
          dup = true;
        }
      if (!dup) table.push_back(e);
    }
  }
  kdb_set_tuning(&g);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_table = table;
  return KDB_OK;
}

kdb_status kdb_autotune(const void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                        int reps, kdb_tuning* out_best, float* out_best_ms, float* h_ms,
                        kdb_stream_t stream) {
  kdb_status s = check_common(n, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  if (n < 2 || reps < 1 || reps > 64 || !d_points || (reinterpret_cast<uintptr_t>(d_points) & 3))
    return KDB_ERR_INVALID_ARGUMENT;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const kdb_tuning cur{g_part_shape.load(), g_rec_shape.load(), g_rec_bits.load()};
  Plan P;
  P.sets.push_back(SetInfo{0u, (uint32_t)n});
  P.total = (uint32_t)n;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split_of(mode);
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  P.part_shape = cur.partition_shape;  // the workspace does not depend on the setting
  P.rec_shape = cur.radix_shape;
  P.rec_bits = cur.digit_bits;
  make_plan(P);
  if (P.too_wide) return KDB_ERR_INVALID_ARGUMENT;
  int dev, sms;
  cudaMemPool_t pool;
  s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  const size_t pts_bytes = (size_t)n * stride_bytes;
  void *copy = nullptr, *ws = nullptr;
  s = pool_alloc(&copy, pts_bytes, pool, st);
  if (s == KDB_OK) s = pool_alloc(&ws, P.bytes, pool, st);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (s == KDB_OK && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess))
    s = KDB_ERR_CUDA;
  // the tuned kernels run only on the list path with at least one global level
  const bool tuned = P.use_lists && !P.act.empty();
  const int np = kPartShapes, nr = kRecShapes, nw = kRecDigitWidths;
  const int combos = np * nr * nw;
  std::vector<float> med(combos, -1.0f);
  std::vector<float> t(reps);
  for (int c = 0; c < combos && s == KDB_OK; ++c) {
    const int ps = c / (nr * nw), rs = (c / nw) % nr, bits = kRecDigitBits[c % nw];
    if (!tuned && (ps != cur.partition_shape || rs != cur.radix_shape || bits != cur.digit_bits)) continue;
    P.part_shape = ps;
    P.rec_shape = rs;
    P.rec_bits = bits;
    for (int r = -1; r < reps && s == KDB_OK; ++r) {  // r = -1: untimed first build
      if (cudaMemcpyAsync(copy, d_points, pts_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaEventRecord(ev[0], st) != cudaSuccess) {
        s = KDB_ERR_CUDA;
        break;
      }
      s = enqueue_build(P, static_cast<unsigned char*>(copy), ws, sms, nullptr, nullptr, st);
      if (cudaEventRecord(ev[1], st) != cudaSuccess && s == KDB_OK) s = KDB_ERR_CUDA;
      const kdb_status f = finish(P, ws, st);
      if (s == KDB_OK) s = f;
      float ms = 0.0f;
      if (s == KDB_OK && cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) s = KDB_ERR_CUDA;
      if (r >= 0) t[r] = ms;
    }
    if (s == KDB_OK) {
      std::sort(t.begin(), t.end());
      med[c] = t[reps / 2];
    }
  }
  int best = -1;
  for (int c = 0; c < combos; ++c)
    if (med[c] >= 0.0f && (best < 0 || med[c] < med[best])) best = c;
  if (s == KDB_OK && best >= 0) {
    const kdb_tuning b{best / (nr * nw), (best / nw) % nr, kRecDigitBits[best % nw]};
    kdb_set_tuning(&b);
    if (tuned)  // kept for later builds of this kind
      put_tuning_entry(TuneEntry{tune_bucket((uint64_t)n), k, stride_bytes, (int)mode, b.partition_shape,
                                 b.radix_shape, b.digit_bits});
    if (out_best) *out_best = b;
    if (out_best_ms) *out_best_ms = med[best];
    if (h_ms) std::copy(med.begin(), med.end(), h_ms);
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  if (copy) cudaFreeAsync(copy, st);
  if (ws) cudaFreeAsync(ws, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && s == KDB_OK) s = KDB_ERR_CUDA;
  cudaGetLastError();
  return s;
}

int kdb_debug_inject_fault(int fault, int64_t arg) {
  const int prev = g_fault;
  g_fault = fault;
  g_fault_arg = arg;
  return prev;
}

size_t kdb_workspace_size(int64_t n, int k, int stride_bytes, kdb_split_mode mode) {
  if (check_common(n, k, stride_bytes) != KDB_OK || check_mode_k(mode, k) != KDB_OK || n <= 1) return 0;
  Plan P;
  P.sets.push_back(SetInfo{0u, (uint32_t)n});
  P.total = (uint32_t)n;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split_of(mode);
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  make_plan(P);
  return P.bytes;
}

kdb_status kdb_build_ex(void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                        void* d_workspace, size_t workspace_bytes, int32_t* d_out_orig_index,
                        uint8_t* d_out_split_dim, kdb_stream_t stream) {
  kdb_status s = check_common(n, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  if (n > 0 && (!d_points || (reinterpret_cast<uintptr_t>(d_points) & 3))) return KDB_ERR_INVALID_ARGUMENT;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n <= 1) {
    if (n == 1) {
      int32_t zero = 0;
      uint8_t z8 = 0;
      if (d_out_orig_index) KDB_CK(cudaMemcpyAsync(d_out_orig_index, &zero, 4, cudaMemcpyHostToDevice, st));
      if (d_out_split_dim) KDB_CK(cudaMemcpyAsync(d_out_split_dim, &z8, 1, cudaMemcpyHostToDevice, st));
      KDB_CK(cudaStreamSynchronize(st));
    }
    return KDB_OK;
  }
  // the memory-lean build, where asked for, or (automatic) where the
  // ordinary workspace does not fit: only for builds without caller
  // workspace or extra outputs
  const int mm = g_memory_mode.load();
  const bool lean_ok = !d_workspace && !d_out_orig_index && !d_out_split_dim && num_levels((uint32_t)n) >= 3;
  if (lean_ok && mm == KDB_MEMORY_LEAN)
    return lean_build(static_cast<unsigned char*>(d_points), n, k, stride_bytes, (int)mode, st);
  const std::shared_ptr<CachedPlan> cp = cached_plan(n, k, stride_bytes, (int)mode);
  if (lean_ok && mm == KDB_MEMORY_AUTO && !cp->P.too_wide && lean_needed(cp->P.bytes))
    return lean_build(static_cast<unsigned char*>(d_points), n, k, stride_bytes, (int)mode, st);
  return run_cached(*cp, static_cast<unsigned char*>(d_points), d_workspace, workspace_bytes, d_out_orig_index,
                    d_out_split_dim, st);
}

kdb_status kdb_build_subtree(void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                             int first_dim, const float* h_root_domain, int32_t* d_out_orig_index,
                             kdb_stream_t stream) {
  kdb_status s = check_common(n, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  const int split = split_of(mode);
  if (first_dim < 0 || first_dim >= k) return KDB_ERR_INVALID_ARGUMENT;
  if (split == KDB_SPLIT_WIDEST_EXTENT && !h_root_domain) return KDB_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!d_points || (reinterpret_cast<uintptr_t>(d_points) & 3))) return KDB_ERR_INVALID_ARGUMENT;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n <= 1) {
    if (n == 1 && d_out_orig_index) {
      int32_t zero = 0;
      KDB_CK(cudaMemcpyAsync(d_out_orig_index, &zero, 4, cudaMemcpyHostToDevice, st));
      KDB_CK(cudaStreamSynchronize(st));
    }
    return KDB_OK;
  }
  Plan P;
  P.sets.push_back(SetInfo{0u, (uint32_t)n});
  P.total = (uint32_t)n;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split;
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  P.dim0 = split == KDB_SPLIT_ROUND_ROBIN ? first_dim : 0;
  if (split == KDB_SPLIT_WIDEST_EXTENT) {
    P.has_domain = true;
    for (int d = 0; d < k; ++d) {
      P.domain[d] = h_root_domain[d];
      P.domain[kMaxK + d] = h_root_domain[k + d];
    }
  }
  return run(P, static_cast<unsigned char*>(d_points), nullptr, 0, d_out_orig_index, nullptr, st);
}

kdb_status kdb_build(void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                     kdb_stream_t stream) {
  return kdb_build_ex(d_points, n, k, stride_bytes, mode, nullptr, 0, nullptr, nullptr, stream);
}

kdb_status kdb_build_noalloc(void* d_points, int64_t n, int k, int stride_bytes,
                             kdb_split_mode mode, kdb_stream_t stream) {
  kdb_status s = check_common(n, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  if (n > KDB_NOALLOC_MAX_POINTS) return KDB_ERR_INVALID_ARGUMENT;
  if (n <= 1) return KDB_OK;
  if (!d_points || (reinterpret_cast<uintptr_t>(d_points) & 3)) return KDB_ERR_INVALID_ARGUMENT;
  Plan P;
  P.sets.push_back(SetInfo{0u, (uint32_t)n});
  P.total = (uint32_t)n;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split_of(mode);
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  make_plan(P);
  if (P.too_wide || P.bytes > KDB_NOALLOC_SCRATCH_BYTES) return KDB_ERR_INVALID_ARGUMENT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return KDB_ERR_CUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return KDB_ERR_CUDA;
  }
  void* ws = nullptr;
  s = noalloc_scratch(dev, &ws);
  if (s != KDB_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = enqueue_build(P, static_cast<unsigned char*>(d_points), ws, sms > 0 ? sms : 1, nullptr,
                    nullptr, st);
  kdb_status f = finish(P, ws, st);
  return s != KDB_OK ? s : f;
}

}  // extern "C"

// ------------------------------------------------- sharded single tree --
namespace kdb {
namespace {
// Common checks of the sharded-build steps and one synchronous run of
// `launch` with a device status word from the pool.
template <class F>
kdb_status dist_run(int64_t n, int k, int stride_bytes, kdb_split_mode mode, int level, uint32_t index_base,
                    kdb_stream_t stream, F launch) {
  kdb_status s = check_common(n, k, stride_bytes);
  if (s == KDB_OK) s = check_mode(mode);
  if (s != KDB_OK) return s;
  if (level < 0 || (1 << level) > kDistMaxDest) return KDB_ERR_INVALID_ARGUMENT;
  if ((uint64_t)index_base + (uint64_t)n > 2147483647ull) return KDB_ERR_INVALID_ARGUMENT;
  int dev, sms;
  cudaMemPool_t pool;
  s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* err = nullptr;
  s = pool_alloc(&err, 4, pool, st);
  if (s != KDB_OK) return s;
  kdb_status r = KDB_OK;
  if (cudaMemsetAsync(err, 0, 4, st) != cudaSuccess || launch(static_cast<uint32_t*>(err), sms, st) != cudaSuccess)
    r = KDB_ERR_CUDA;
  uint32_t h_err = 0;
  if (r == KDB_OK && cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) r = KDB_ERR_CUDA;
  cudaFreeAsync(err, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) r = KDB_ERR_CUDA;
  if (r != KDB_OK) {
    cudaGetLastError();
    return r;
  }
  return (h_err & ERR_INTERNAL) ? KDB_ERR_INTERNAL : KDB_OK;
}

DistArgs dist_args(const void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode, const int32_t* d_tags,
                   int level, uint32_t index_base) {
  DistArgs a{};
  a.pts = static_cast<const unsigned char*>(d_points);
  a.n = (uint32_t)n;
  a.k = k;
  a.stride = stride_bytes;
  a.ctype = ctype_of((int)mode);
  a.tags = const_cast<int32_t*>(d_tags);
  a.first = full_nodes(level);
  a.nodes = 1u << level;
  a.index_base = index_base;
  return a;
}
}  // namespace
}  // namespace kdb

extern "C" {

kdb_status kdb_dist_histogram(const void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                              const int32_t* d_tags, int level, const uint8_t* d_node_dim,
                              const uint64_t* d_node_prefix, int prefix_bits, uint32_t index_base,
                              uint32_t* d_hist, kdb_stream_t stream) {
  if (prefix_bits < 0 || prefix_bits > 56 || prefix_bits % 8 || !d_hist || !d_node_dim || !d_node_prefix ||
      (n > 0 && (!d_points || !d_tags)))
    return KDB_ERR_INVALID_ARGUMENT;
  return dist_run(n, k, stride_bytes, mode, level, index_base, stream,
                  [&](uint32_t* err, int sms, cudaStream_t st) -> cudaError_t {
                    DistArgs a = dist_args(d_points, n, k, stride_bytes, mode, d_tags, level, index_base);
                    a.node_dim = d_node_dim;
                    a.prefix = d_node_prefix;
                    a.prefix_bits = prefix_bits;
                    a.hist = d_hist;
                    a.err = err;
                    cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)a.nodes * 256 * 4, st);
                    return e != cudaSuccess ? e : launch_dist_hist(a, sms, st);
                  });
}

kdb_status kdb_dist_box(const void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                        const int32_t* d_tags, int level, uint32_t* d_box, kdb_stream_t stream) {
  if (!d_box || (n > 0 && (!d_points || !d_tags))) return KDB_ERR_INVALID_ARGUMENT;
  return dist_run(n, k, stride_bytes, mode, level, 0, stream,
                  [&](uint32_t* err, int sms, cudaStream_t st) -> cudaError_t {
                    DistArgs a = dist_args(d_points, n, k, stride_bytes, mode, d_tags, level, 0);
                    a.box = d_box;
                    a.err = err;
                    std::vector<uint32_t> init((size_t)a.nodes * 2 * k);
                    for (size_t i = 0; i < init.size(); ++i) init[i] = (i / k) % 2 == 0 ? 0xFFFFFFFFu : 0u;
                    cudaError_t e = cudaMemcpyAsync(d_box, init.data(), init.size() * 4, cudaMemcpyHostToDevice, st);
                    return e != cudaSuccess ? e : launch_dist_box(a, sms, st);
                  });
}

kdb_status kdb_dist_assign(const void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                           int32_t* d_tags, int level, const uint8_t* d_node_dim, const uint64_t* d_pivot,
                           uint32_t index_base, int64_t* d_pinned, kdb_stream_t stream) {
  if (!d_node_dim || !d_pivot || !d_pinned || (n > 0 && (!d_points || !d_tags))) return KDB_ERR_INVALID_ARGUMENT;
  return dist_run(n, k, stride_bytes, mode, level, index_base, stream,
                  [&](uint32_t* err, int sms, cudaStream_t st) -> cudaError_t {
                    DistArgs a = dist_args(d_points, n, k, stride_bytes, mode, d_tags, level, index_base);
                    a.node_dim = d_node_dim;
                    a.pivot = d_pivot;
                    a.pinned = d_pinned;
                    a.err = err;
                    return launch_dist_assign(a, sms, st);
                  });
}

kdb_status kdb_dist_partition(const void* d_points, int64_t n, int stride_bytes, const int32_t* d_tags,
                              int32_t first_node, int num_dest, uint32_t index_base, void* d_out_points,
                              uint32_t* d_out_index, int64_t* h_counts, kdb_stream_t stream) {
  if (num_dest < 1 || num_dest > kDistMaxDest || first_node < 0 || !h_counts) return KDB_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!d_points || !d_tags || !d_out_points || !d_out_index)) return KDB_ERR_INVALID_ARGUMENT;
  if (n < 0 || n > 2147483647LL || stride_bytes < 4 || stride_bytes % 4 ||
      (uint64_t)index_base + (uint64_t)n > 2147483647ull)
    return KDB_ERR_INVALID_ARGUMENT;
  for (int j = 0; j < num_dest; ++j) h_counts[j] = 0;
  if (n == 0) return KDB_OK;
  int dev, sms;
  cudaMemPool_t pool;
  kdb_status s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DistArgs a{};
  a.pts = static_cast<const unsigned char*>(d_points);
  a.n = (uint32_t)n;
  a.stride = stride_bytes;
  a.tags = const_cast<int32_t*>(d_tags);
  a.first = (uint32_t)first_node;
  a.nodes = (uint32_t)num_dest;
  a.index_base = index_base;
  a.out_pts = static_cast<unsigned char*>(d_out_points);
  a.out_index = d_out_index;
  const uint32_t blocks = dist_blocks(a.n, sms);
  const size_t cnt = (size_t)blocks * num_dest;
  void* ws = nullptr;
  s = pool_alloc(&ws, cnt * 8 + 4, pool, st);
  if (s != KDB_OK) return s;
  a.block_counts = static_cast<uint32_t*>(ws);
  a.err = a.block_counts + 2 * cnt;
  std::vector<uint32_t> h(cnt);
  kdb_status r = KDB_OK;
  if (cudaMemsetAsync(a.err, 0, 4, st) != cudaSuccess || launch_dist_count(a, blocks, st) != cudaSuccess ||
      cudaMemcpyAsync(h.data(), a.block_counts, cnt * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    r = KDB_ERR_CUDA;
  } else {
    // exclusive offsets: destination-major, then block order (a stable partition)
    std::vector<uint32_t> off(cnt);
    uint64_t run = 0;
    for (int j = 0; j < num_dest; ++j) {
      const uint64_t first = run;
      for (uint32_t b = 0; b < blocks; ++b) {
        off[(size_t)b * num_dest + j] = (uint32_t)run;
        run += h[(size_t)b * num_dest + j];
      }
      h_counts[j] = (int64_t)(run - first);
    }
    a.block_offsets = a.block_counts + cnt;
    uint32_t h_err = 0;
    if (cudaMemcpyAsync(const_cast<uint32_t*>(a.block_offsets), off.data(), cnt * 4, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        launch_dist_scatter(a, blocks, st) != cudaSuccess ||
        cudaMemcpyAsync(&h_err, a.err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      r = KDB_ERR_CUDA;
    else if (h_err & ERR_INTERNAL)
      r = KDB_ERR_INTERNAL;
  }
  cudaFreeAsync(ws, st);
  cudaStreamSynchronize(st);
  if (r == KDB_ERR_CUDA) cudaGetLastError();
  return r;
}

kdb_status kdb_build_batched(void* d_points, const int64_t* h_offsets, int num_sets, int k,
                             int stride_bytes, kdb_split_mode mode, kdb_stream_t stream) {
  if (num_sets < 0 || (num_sets > 0 && !h_offsets)) return KDB_ERR_INVALID_ARGUMENT;
  if (num_sets == 0) return KDB_OK;
  if (h_offsets[0] != 0) return KDB_ERR_INVALID_ARGUMENT;
  const int64_t total = h_offsets[num_sets];
  kdb_status s = check_common(total, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  if (total > 0 && (!d_points || (reinterpret_cast<uintptr_t>(d_points) & 3))) return KDB_ERR_INVALID_ARGUMENT;
  Plan P;
  P.sets.reserve(num_sets);
  for (int b = 0; b < num_sets; ++b) {
    if (h_offsets[b + 1] < h_offsets[b]) return KDB_ERR_INVALID_ARGUMENT;
    P.sets.push_back(SetInfo{(uint32_t)h_offsets[b], (uint32_t)(h_offsets[b + 1] - h_offsets[b])});
  }
  if (total <= 1) return KDB_OK;
  P.total = (uint32_t)total;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split_of(mode);
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  return run(P, static_cast<unsigned char*>(d_points), nullptr, 0, nullptr, nullptr,
             reinterpret_cast<cudaStream_t>(stream));
}

namespace kdb {
namespace {
// The sets of a batched call as a plan (make_plan not yet run); checks the
// arguments shared by the batched entry points.
kdb_status batched_sets(Plan& P, const int64_t* h_offsets, int num_sets, int k, int stride_bytes,
                        kdb_split_mode mode) {
  if (num_sets < 1 || !h_offsets || h_offsets[0] != 0) return KDB_ERR_INVALID_ARGUMENT;
  const int64_t total = h_offsets[num_sets];
  kdb_status s = check_common(total, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  P.sets.reserve(num_sets);
  for (int b = 0; b < num_sets; ++b) {
    if (h_offsets[b + 1] < h_offsets[b]) return KDB_ERR_INVALID_ARGUMENT;
    P.sets.push_back(SetInfo{(uint32_t)h_offsets[b], (uint32_t)(h_offsets[b + 1] - h_offsets[b])});
  }
  P.total = (uint32_t)total;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split_of(mode);
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  return KDB_OK;
}
}  // namespace
}  // namespace kdb

size_t kdb_batched_workspace_size(const int64_t* h_offsets, int num_sets, int k, int stride_bytes,
                                  kdb_split_mode mode) {
  kdb::Plan P;
  if (kdb::batched_sets(P, h_offsets, num_sets, k, stride_bytes, mode) != KDB_OK || P.total <= 1)
    return 0;
  kdb::make_plan(P);
  return P.too_wide ? 0 : P.bytes;
}

kdb_status kdb_build_batched_async(void* d_points, const int64_t* h_offsets, int num_sets, int k,
                                   int stride_bytes, kdb_split_mode mode, void* d_workspace,
                                   size_t workspace_bytes, uint32_t* d_error_word,
                                   kdb_stream_t stream) {
  kdb::Plan P;
  kdb_status s = kdb::batched_sets(P, h_offsets, num_sets, k, stride_bytes, mode);
  if (s != KDB_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (P.total <= 1) {
    if (d_error_word) KDB_CK(cudaMemsetAsync(d_error_word, 0, 4, st));
    return KDB_OK;
  }
  if (!d_points || (reinterpret_cast<uintptr_t>(d_points) & 3)) return KDB_ERR_INVALID_ARGUMENT;
  kdb::make_plan(P);
  if (P.too_wide) return KDB_ERR_INVALID_ARGUMENT;
  if (!d_workspace || workspace_bytes < P.bytes || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
    return KDB_ERR_INVALID_ARGUMENT;
  int dev, sms;
  cudaMemPool_t pool;
  s = kdb::device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  s = kdb::enqueue_build(P, static_cast<unsigned char*>(d_points), d_workspace, sms, nullptr, nullptr,
                         st);
  if (s != KDB_OK) return s;
  if (d_error_word)
    KDB_CK(cudaMemcpyAsync(d_error_word, kdb::at<uint32_t>(d_workspace, P.o_err), 4,
                           cudaMemcpyDeviceToDevice, st));
  return KDB_OK;
}

kdb_status kdb_error_word_status(uint32_t word) {
  if (word & kdb::ERR_NAN) return KDB_ERR_NAN_INPUT;
  if (word & kdb::ERR_TIMEOUT) return KDB_ERR_TIMEOUT;
  if (word) return KDB_ERR_INTERNAL;
  return KDB_OK;
}

kdb_status kdb_plan_create(const int64_t* h_offsets, int num_sets, int k, int stride_bytes,
                           kdb_split_mode mode, kdb_plan* out_plan) {
  using kdb::PlanObj;
  if (!out_plan) return KDB_ERR_INVALID_ARGUMENT;
  *out_plan = nullptr;
  if (num_sets < 1 || !h_offsets || h_offsets[0] != 0) return KDB_ERR_INVALID_ARGUMENT;
  const int64_t total = h_offsets[num_sets];
  kdb_status s = kdb::check_common(total, k, stride_bytes);
  if (s == KDB_OK) s = kdb::check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  PlanObj* po = new (std::nothrow) PlanObj();
  if (!po) return KDB_ERR_OUT_OF_MEMORY;
  kdb::Plan& P = po->P;
  for (int b = 0; b < num_sets; ++b) {
    if (h_offsets[b + 1] < h_offsets[b]) {
      delete po;
      return KDB_ERR_INVALID_ARGUMENT;
    }
    P.sets.push_back(kdb::SetInfo{(uint32_t)h_offsets[b], (uint32_t)(h_offsets[b + 1] - h_offsets[b])});
  }
  P.total = (uint32_t)total;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split_of(mode);
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  po->trivial = total <= 1;
  if (po->trivial) {
    *out_plan = reinterpret_cast<kdb_plan>(po);
    return KDB_OK;
  }
  kdb::make_plan(P);
  cudaMemPool_t pool;
  s = P.too_wide ? KDB_ERR_INVALID_ARGUMENT : kdb::device_setup(&po->dev, &pool, &po->sms);
  void* pts = nullptr;
  if (s == KDB_OK && (cudaMalloc(&po->ws, P.bytes) != cudaSuccess ||
                      cudaMallocHost(reinterpret_cast<void**>(&po->h_err), 4) != cudaSuccess)) {
    cudaGetLastError();
    s = KDB_ERR_OUT_OF_MEMORY;
  }
  if (s == KDB_OK) s = kdb::upload_tables(P, po->ws, nullptr, true);
  // one build on all-zero points outside any capture: loads every kernel and
  // sets its attributes, so that later enqueues only launch
  if (s == KDB_OK) {
    if (cudaMalloc(&pts, (size_t)total * stride_bytes) != cudaSuccess ||
        cudaMemset(pts, 0, (size_t)total * stride_bytes) != cudaSuccess) {
      cudaGetLastError();
      s = KDB_ERR_OUT_OF_MEMORY;
    }
  }
  if (s == KDB_OK) {
    s = kdb::enqueue_build(P, static_cast<unsigned char*>(pts), po->ws, po->sms, nullptr, nullptr,
                           nullptr, true);
    kdb_status f = kdb::finish(P, po->ws, nullptr);
    if (s == KDB_OK) s = f;
  }
  if (pts) cudaFree(pts);
  if (s != KDB_OK) {
    kdb_plan_destroy(reinterpret_cast<kdb_plan>(po));
    return s;
  }
  *out_plan = reinterpret_cast<kdb_plan>(po);
  return KDB_OK;
}

kdb_status kdb_plan_enqueue(kdb_plan plan, void* d_points, kdb_stream_t stream) {
  kdb::PlanObj* po = reinterpret_cast<kdb::PlanObj*>(plan);
  if (!po) return KDB_ERR_INVALID_ARGUMENT;
  if (po->trivial) return KDB_OK;
  if (!d_points || (reinterpret_cast<uintptr_t>(d_points) & 3)) return KDB_ERR_INVALID_ARGUMENT;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != po->dev) {
    cudaGetLastError();
    return KDB_ERR_INVALID_ARGUMENT;
  }
  return kdb::enqueue_build(po->P, static_cast<unsigned char*>(d_points), po->ws, po->sms, nullptr,
                            nullptr, reinterpret_cast<cudaStream_t>(stream), true);
}

kdb_status kdb_plan_status(kdb_plan plan, kdb_stream_t stream) {
  kdb::PlanObj* po = reinterpret_cast<kdb::PlanObj*>(plan);
  if (!po) return KDB_ERR_INVALID_ARGUMENT;
  if (po->trivial) return KDB_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(po->h_err, kdb::at<uint32_t>(po->ws, po->P.o_err), 4, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return KDB_ERR_CUDA;
  }
  const uint32_t e = *po->h_err;
  if (e & kdb::ERR_NAN) return KDB_ERR_NAN_INPUT;
  if (e & kdb::ERR_TIMEOUT) return KDB_ERR_TIMEOUT;
  if (e & kdb::ERR_INTERNAL) return KDB_ERR_INTERNAL;
  return KDB_OK;
}

size_t kdb_plan_workspace_bytes(kdb_plan plan) {
  const kdb::PlanObj* po = reinterpret_cast<const kdb::PlanObj*>(plan);
  return po && !po->trivial ? po->P.bytes : 0;
}

void kdb_plan_destroy(kdb_plan plan) {
  kdb::PlanObj* po = reinterpret_cast<kdb::PlanObj*>(plan);
  if (!po) return;
  if (po->ws) cudaFree(po->ws);
  if (po->h_err) cudaFreeHost(po->h_err);
  cudaGetLastError();
  delete po;
}

kdb_status kdb_build_host(void* h_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                          kdb_stream_t stream) {
  kdb_status s = check_common(n, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  if (n <= 1) return KDB_OK;
  if (!h_points) return KDB_ERR_INVALID_ARGUMENT;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev, sms;
  cudaMemPool_t pool;
  s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  Plan P;
  P.sets.push_back(SetInfo{0u, (uint32_t)n});
  P.total = (uint32_t)n;
  P.k = k;
  P.stride = stride_bytes;
  P.mode = split_of(mode);
  P.ctype = ctype_of(mode);
  P.mode_arg = (int)mode;
  make_plan(P);
  if (P.too_wide) return KDB_ERR_INVALID_ARGUMENT;
  // Records without payload in page-locked memory that this device can
  // address: every record the build writes is rebuilt from its entry, so the
  // kernels read the caller's records and write the tree straight into them
  // (over the host link), with no device copy of the records at all.
  P.placement = g_placement.load();
  if (P.can_direct && P.placement == KDB_PLACEMENT_AUTO &&
      (reinterpret_cast<uintptr_t>(h_points) & 3) == 0) {
    cudaPointerAttributes pa;
    void* mapped = nullptr;
    if (cudaPointerGetAttributes(&pa, h_points) == cudaSuccess && pa.type == cudaMemoryTypeHost)
      mapped = pa.devicePointer;
    cudaGetLastError();
    if (mapped) {
      void* ws = nullptr;
      s = pool_alloc(&ws, P.bytes, pool, st);
      if (s == KDB_OK) s = enqueue_build(P, static_cast<unsigned char*>(mapped), ws, sms, nullptr, nullptr, st);
      const kdb_status f = ws ? finish(P, ws, st) : KDB_OK;
      if (s == KDB_OK) s = f;
      if (ws) cudaFreeAsync(ws, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        if (s == KDB_OK) s = KDB_ERR_CUDA;
      }
      return s;
    }
  }
  const size_t bytes = (size_t)n * stride_bytes;
  void* d = nullptr;
  void* ws = nullptr;
  s = pool_alloc(&d, bytes, pool, st);
  if (s == KDB_OK) s = pool_alloc(&ws, P.bytes, pool, st);
  // the records go to the device in chunks on a second stream, so that the
  // prepass of each chunk overlaps the copy of the next
  HostFeed feed;
  feed.h = static_cast<const unsigned char*>(h_points);
  feed.chunks = (int)std::min<size_t>(8, std::max<size_t>(1, bytes >> 26));  // >= 64 MiB a chunk
  cudaEvent_t ready = nullptr;
  bool made = s == KDB_OK && cudaStreamCreateWithFlags(&feed.cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess;
  for (int c = 0; made && c < feed.chunks; ++c)
    made = cudaEventCreateWithFlags(&feed.ev[c], cudaEventDisableTiming) == cudaSuccess;
  if (s == KDB_OK && !made) s = KDB_ERR_CUDA;
  if (s == KDB_OK) {
    // the copies may start once the allocations on `st` are done
    if (cudaEventRecord(ready, st) != cudaSuccess || cudaStreamWaitEvent(feed.cs, ready, 0) != cudaSuccess)
      s = KDB_ERR_CUDA;
  }
  if (s == KDB_OK) s = enqueue_build(P, static_cast<unsigned char*>(d), ws, sms, nullptr, nullptr, st, false,
                                     &feed);
  if (s == KDB_OK) s = finish(P, ws, st);
  if (s == KDB_OK &&
      cudaMemcpyAsync(h_points, d, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    s = KDB_ERR_CUDA;
  if (s != KDB_OK) cudaGetLastError();
  if (feed.cs) cudaStreamSynchronize(feed.cs);  // no copy left in flight
  if (ws) cudaFreeAsync(ws, st);
  if (d) cudaFreeAsync(d, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    if (s == KDB_OK) s = KDB_ERR_CUDA;
  }
  for (int c = 0; c < feed.chunks; ++c)
    if (feed.ev[c]) cudaEventDestroy(feed.ev[c]);
  if (ready) cudaEventDestroy(ready);
  if (feed.cs) cudaStreamDestroy(feed.cs);
  return s;
}

kdb_status kdb_validate(const void* d_points, int64_t n, int k, int stride_bytes,
                        kdb_split_mode mode, int64_t* h_first_bad_node, kdb_stream_t stream) {
  kdb_status s = check_common(n, k, stride_bytes);
  if (s == KDB_OK) s = check_mode_k(mode, k);
  if (s != KDB_OK) return s;
  if (h_first_bad_node) *h_first_bad_node = -1;
  if (n <= 1) return KDB_OK;
  if (!d_points || (reinterpret_cast<uintptr_t>(d_points) & 3)) return KDB_ERR_INVALID_ARGUMENT;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev, sms;
  cudaMemPool_t pool;
  s = device_setup(&dev, &pool, &sms);
  if (s != KDB_OK) return s;
  const uint32_t N = (uint32_t)n;
  const bool widest = split_of(mode) == KDB_SPLIT_WIDEST_EXTENT;
  const bool tight = split_of(mode) == KDB_SPLIT_WIDEST_TIGHT;
  const int ctype = ctype_of(mode);
  const int L = num_levels(N);
  // single-set tables for the dimension pass (widest mode)
  std::vector<ActiveEntry> act(std::max(1, L - 1));
  for (int l = 0; l < (int)act.size(); ++l) {
    act[l].set = 0;
    act[l].base = 0;
    act[l].next = (l + 1 < (int)act.size()) ? 0 : -1;
    act[l].box0 = 0;
  }
  const size_t box_bytes = widest ? ((size_t)1 << std::max(0, L - 1)) * 2 * k * 4 : 0;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t a = o;
    o = align256(o + b);
    return a;
  };
  const size_t o_bad = take(4), o_err = take(4), o_bbox = take(2 * k * 4), o_sets = take(sizeof(SetInfo)),
               o_act = take(act.size() * sizeof(ActiveEntry)), o_dims = take(widest || tight ? N : 0),
               o_bA = take(box_bytes), o_bB = take(box_bytes),
               o_tbox = take(tight ? (size_t)N * 2 * k * 4 : 0);
  void* ws = nullptr;
  s = pool_alloc(&ws, o, pool, st);
  if (s != KDB_OK) return s;
  uint32_t* bad = at<uint32_t>(ws, o_bad);
  kdb_status result = KDB_OK;
  do {
    if (cudaMemsetAsync(bad, 0xFF, 4, st) != cudaSuccess) { result = KDB_ERR_CUDA; break; }
    uint8_t* dims = nullptr;
    if (widest) {
      SetInfo one{0u, N};
      std::vector<uint32_t> init(2 * k);
      for (int d = 0; d < k; ++d) {
        init[d] = 0xFFFFFFFFu;
        init[k + d] = 0u;
      }
      dims = at<uint8_t>(ws, o_dims);
      if (cudaMemcpyAsync(at<void>(ws, o_sets), &one, sizeof one, cudaMemcpyHostToDevice, st) ||
          cudaMemcpyAsync(at<void>(ws, o_act), act.data(), act.size() * sizeof(ActiveEntry),
                          cudaMemcpyHostToDevice, st) ||
          cudaMemcpyAsync(at<void>(ws, o_bbox), init.data(), init.size() * 4,
                          cudaMemcpyHostToDevice, st) ||
          cudaMemsetAsync(at<void>(ws, o_err), 0, 4, st) || cudaMemsetAsync(dims, 0, N, st)) {
        result = KDB_ERR_CUDA;
        break;
      }
      PrepassArgs pa{};
      pa.pts = static_cast<const unsigned char*>(d_points);
      pa.total = N;
      pa.k = k;
      pa.stride = stride_bytes;
      pa.sets = at<SetInfo>(ws, o_sets);
      pa.nsets = 1;
      pa.bbox = at<uint32_t>(ws, o_bbox);
      pa.err = at<uint32_t>(ws, o_err);
      if (launch_prepass(pa, sms, st) != cudaSuccess) { result = KDB_ERR_CUDA; break; }
      ActiveEntry* d_act = at<ActiveEntry>(ws, o_act);
      if (launch_widest_root(pa.sets, d_act, 1, pa.bbox, k, at<float>(ws, o_bA), dims, false, st) !=
          cudaSuccess) { result = KDB_ERR_CUDA; break; }
      for (int l = 0; l + 1 < L; ++l) {
        WidestArgs wa{};
        wa.x.sets = pa.sets;
        wa.x.act = d_act + l;
        wa.x.act_next = l + 1 < (int)act.size() ? d_act + l + 1 : nullptr;
        wa.x.nact = 1;
        wa.x.l = l;
        wa.x.rb = 0;
        wa.x.err = at<uint32_t>(ws, o_err);
        wa.pts = pa.pts;
        wa.k = k;
        wa.stride = stride_bytes;
        wa.perm = nullptr;
        wa.boxes_in = at<float>(ws, (l & 1) ? o_bB : o_bA);
        wa.boxes_out = at<float>(ws, (l & 1) ? o_bA : o_bB);
        wa.dims = dims;
        wa.total_threads = 1u << l;
        if (launch_widest_children(wa, st) != cudaSuccess) { result = KDB_ERR_CUDA; break; }
      }
      if (result != KDB_OK) break;
    }
    if (tight) {
      dims = at<uint8_t>(ws, o_dims);
      if (launch_tight_validate_dims(static_cast<const unsigned char*>(d_points), N, k, stride_bytes,
                                     at<uint32_t>(ws, o_tbox), dims, ctype, st) != cudaSuccess) {
        result = KDB_ERR_CUDA;
        break;
      }
    }
    g_launches += widest || tight ? L + 1 : 1;  // prepass / boxes, dimension passes, check
    if (launch_validate(static_cast<const unsigned char*>(d_points), N, k, stride_bytes, mode, dims,
                        bad, st) != cudaSuccess) { result = KDB_ERR_CUDA; break; }
    uint32_t h_bad = 0xFFFFFFFFu;
    if (cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { result = KDB_ERR_CUDA; break; }
    if (h_bad != 0xFFFFFFFFu) {
      if (h_first_bad_node) *h_first_bad_node = (int64_t)h_bad;
      result = KDB_ERR_NOT_A_KD_TREE;
    }
  } while (0);
  if (result == KDB_ERR_CUDA) cudaGetLastError();
  cudaFreeAsync(ws, st);
  cudaStreamSynchronize(st);
  return result;
}

}  // extern "C"
extern "C" {

kdb_memory_mode kdb_set_memory_mode(kdb_memory_mode m) {
  if (m != KDB_MEMORY_AUTO && m != KDB_MEMORY_FAST && m != KDB_MEMORY_LEAN)
    return (kdb_memory_mode)kdb::g_memory_mode.load();
  return (kdb_memory_mode)kdb::g_memory_mode.exchange(m);
}

size_t kdb_lean_workspace_size(int64_t n, int k, int stride_bytes, kdb_split_mode mode) {
  if (check_common(n, k, stride_bytes) != KDB_OK || check_mode_k(mode, k) != KDB_OK) return 0;
  int dev, sms;
  cudaMemPool_t pool;
  if (device_setup(&dev, &pool, &sms) != KDB_OK) sms = 152;  // no GPU: the size for a GB300
  const kdb::LeanPlan L = kdb::lean_plan(n, k, stride_bytes, (int)mode, sms);
  return L.g ? L.bytes : 0;
}

}  // extern "C"
