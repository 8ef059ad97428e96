/*
 * kdb.h -- C ABI of the GB300 (sm_103a) left-balanced k-d tree builder.
 *
 * The operation is the one defined in Wald, "GPU-friendly, Parallel, and
 * (Almost-)In-Place Construction of Left-Balanced k-d Trees" (arXiv
 * 2211.00120): given N k-dimensional points, permute them so that the array
 * is a left-balanced, complete k-d tree in level order -- node i at record i,
 * children of i at 2i+1 and 2i+2 (Sec. 2) -- where every node is >= all nodes
 * of its left subtree and <= all nodes of its right subtree in its split
 * dimension (Sec. 1).  The split dimension is level mod k (round robin,
 * Sec. 2) or the dimension of widest extent of the subtree's domain, the
 * scene box clipped by the ancestors' planes (split-widest, Sec. 6).
 *
 * The build follows the paper's method: O(log N) iterations, each a
 * whole-array sort by (subtree tag, split coordinate) and a per-point tag
 * update (Sec. 3), followed by one placement of the records (Sec. 3.2, 7.1).
 *
 * Conventions shared by every call:
 *   - Records: N records of stride_bytes each, the k coordinates are float32
 *     (or int32 / uint32, with KDB_COORDS_INT32 / KDB_COORDS_UINT32 in the
 *     mode argument) at byte offsets
 *     0, 4, ..., 4(k-1); bytes after 4k are payload that is
 *     moved with the record and never read as a coordinate.  1 <= k <= 8,
 *     stride_bytes >= 4k and a multiple of 4, the base 4-byte aligned.
 *   - 0 <= N <= 2^31 - 1 (the paper's tags are 32-bit ints, Sec. 3).
 *   - Ties: points are ordered by (coordinate, original index), -0.0 before
 *     +0.0, so the tree is unique (the paper's less() in Sec. 3.1 leaves equal
 *     keys unordered).  NaN coordinates are rejected.
 *   - Device pointers are CUDA device (or managed) memory owned by the
 *     caller; "h_" pointers are host memory.  The library never frees caller
 *     memory and keeps no pointer to it after a call returns.
 *   - Streams: work is ordered on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream).  A build may run parts of its work side by side on
 *     streams of its own, forked from `stream` and joined back to it before
 *     anything that follows (not while `stream` is being captured into a
 *     graph), so the order seen from `stream` is unchanged.  Calls that return
 *     device-detected errors synchronise the stream before returning, as
 *     stated per call.
 *   - Errors: argument errors return KDB_ERR_INVALID_ARGUMENT before anything
 *     is enqueued.  If a device error is detected (NaN input, a bounded wait
 *     that ran out, an internal consistency check) the records are left
 *     untouched: the final placement is skipped on the device.
 *   - Thread safety: calls on different streams may run concurrently; each
 *     call uses its own workspace.
 */
#ifndef KDB_H
#define KDB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KDB_API __attribute__((visibility("default")))
#else
#define KDB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream. */
typedef struct CUstream_st* kdb_stream_t;

typedef enum {
  KDB_SPLIT_ROUND_ROBIN = 0,   /* dimension = level mod k (Sec. 2) */
  KDB_SPLIT_WIDEST_EXTENT = 1, /* widest side of the clipped domain (Sec. 6) */
  /* widest side of the subtree's tight bounding box, the box of its own
     points (a rule the paper does not have; Sec. 6 uses the domain instead):
     same extent arithmetic, corners under the strict order.  k <= 3 only;
     other k return KDB_ERR_INVALID_ARGUMENT. */
  KDB_SPLIT_WIDEST_TIGHT = 2
} kdb_split_mode;

/*
 * Coordinate type, OR'ed into the mode argument of every call (build,
 * batched, plans, server, validate); at most one of the two:
 *   KDB_COORDS_INT32   the k coordinates are int32 instead of float32,
 *                      ordered as signed integers -- the paper's int1 / int2
 *                      data (Table 1, Sec. 5);
 *   KDB_COORDS_UINT32  they are uint32, ordered as unsigned integers (another
 *                      scalar type of the templated builder of Sec. 7.2).
 * Tight-box extents of integer coordinates are exact 64-bit differences.
 * The clipped domain rule (KDB_SPLIT_WIDEST_EXTENT) clips float boxes and is
 * float32 only: with either flag it returns KDB_ERR_INVALID_ARGUMENT, as does
 * a mode with both flags.  No NaN check applies to integer coordinates.
 */
#define KDB_COORDS_INT32 0x100
#define KDB_COORDS_UINT32 0x200

typedef enum {
  KDB_OK = 0,
  KDB_ERR_INVALID_ARGUMENT = 1,
  KDB_ERR_OUT_OF_MEMORY = 2,
  KDB_ERR_CUDA = 3,
  KDB_ERR_NAN_INPUT = 4,
  KDB_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
  KDB_ERR_NOT_A_KD_TREE = 6,  /* returned by kdb_validate only */
  KDB_ERR_INTERNAL = 7        /* a device-side consistency check failed */
} kdb_status;

/* Static, NUL-terminated description of a status code. */
KDB_API const char* kdb_status_string(kdb_status status);

/* Library version as major*10000 + minor*100 + patch. */
KDB_API int kdb_version(void);

/*
 * kdb_build -- build the tree in place (Sec. 3.2, parallelKDTreeBuild).
 *   d_points      device, in/out: N records, permuted in place into level
 *                 order.
 *   n, k, stride_bytes, mode: as above.
 * Allocates its workspace from a library-owned stream-ordered pool, runs on
 * `stream`, synchronises `stream` and returns the device status.  N <= 1
 * returns KDB_OK immediately.
 */
KDB_API kdb_status kdb_build(void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                     kdb_stream_t stream);

/*
 * kdb_build_subtree -- build the subtree below one node of a larger tree, in
 * place, in the subtree's own level order (its root at record 0, children of
 * record i at 2i+1 and 2i+2).  A subtree of a left-balanced complete tree is
 * itself one (Sec. 2, Observation 3), so this is kdb_build with the split
 * rule continued from the node: used by the sharded single-tree build, where
 * the top levels are split across GPUs and each GPU builds one subtree.
 *   d_points, n, k, stride_bytes, mode: as for kdb_build.  Ties are broken
 *                 by the records' order in d_points, so the caller passes them
 *                 in ascending original index.
 *   first_dim     round robin: the subtree's root splits in dimension
 *                 first_dim and level l below it in (first_dim + l) mod k
 *                 (the root's depth in the larger tree, mod k); 0 <= first_dim
 *                 < k; ignored by the other rules.
 *   h_root_domain host, 2k floats (lower corner, then upper corner): the
 *                 root's domain, the scene box clipped by the planes of its
 *                 ancestors (Sec. 6); required by KDB_SPLIT_WIDEST_EXTENT,
 *                 ignored by the other rules (the tight box needs no input).
 *   d_out_orig_index device int32[N] or NULL: position in d_points (on entry)
 *                 of the record that ends up at each node.
 * Synchronises `stream`; errors as for kdb_build.
 */
KDB_API kdb_status kdb_build_subtree(void* d_points, int64_t n, int k, int stride_bytes,
                                     kdb_split_mode mode, int first_dim, const float* h_root_domain,
                                     int32_t* d_out_orig_index, kdb_stream_t stream);

/*
 * kdb_workspace_size -- bytes of device workspace kdb_build_ex needs for
 * this problem (0 for N <= 1).  Returns 0 for invalid arguments too.
 */
KDB_API size_t kdb_workspace_size(int64_t n, int k, int stride_bytes, kdb_split_mode mode);

/*
 * kdb_build_ex -- kdb_build with caller-provided workspace and extra outputs.
 *   d_workspace     device, >= kdb_workspace_size() bytes, 256-byte aligned,
 *                   or NULL to use the library pool.  Owned by the caller; its
 *                   contents on entry do not matter.
 *   d_out_orig_index  device int32[N] or NULL: original index (position in
 *                   the input) of the record stored at each node.
 *   d_out_split_dim device uint8[N] or NULL: split dimension of each node.
 * Synchronises `stream` and returns the device status.
 */
KDB_API kdb_status kdb_build_ex(void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                        void* d_workspace, size_t workspace_bytes, int32_t* d_out_orig_index,
                        uint8_t* d_out_split_dim, kdb_stream_t stream);

/*
 * kdb_build_batched -- build num_sets independent trees in one pipeline.
 *   d_points    device, in/out: the sets back to back; set b is records
 *               [h_offsets[b], h_offsets[b+1]) and is permuted in place into
 *               its own level-order tree.
 *   h_offsets   host int64[num_sets+1], non-decreasing, h_offsets[0] = 0,
 *               every set size <= 2^31 - 1.
 * Ties use the index within the set, so every set's output equals a
 * kdb_build of that set alone.  Synchronises `stream`.
 */
KDB_API kdb_status kdb_build_batched(void* d_points, const int64_t* h_offsets, int num_sets, int k,
                             int stride_bytes, kdb_split_mode mode, kdb_stream_t stream);

/*
 * kdb_build_batched_async -- kdb_build_batched that only enqueues: the same
 * build of num_sets independent trees (h_offsets, k, stride_bytes, mode as
 * for kdb_build_batched), with caller workspace and no synchronisation.
 * The paper has no batched build; each set is the paper's build (Sec. 3.2)
 * and its output equals a kdb_build of that set alone.
 *   d_workspace     device, >= kdb_batched_workspace_size() bytes for the
 *                   same arguments, 256-byte aligned, owned by the caller;
 *                   its contents on entry do not matter.  A call uses it
 *                   until the enqueued work has finished.
 *   d_error_word    device uint32 or NULL: receives, in stream order, the
 *                   build's device error flags (0 = success); map it with
 *                   kdb_error_word_status.
 * Host memory is read only during the call (the set table is copied into
 * the workspace on `stream`), so h_offsets may be reused at once.  Returns
 * argument and launch errors; device errors (NaN input, timeouts) arrive in
 * d_error_word, and then every set's records are left as they were.
 */
KDB_API size_t kdb_batched_workspace_size(const int64_t* h_offsets, int num_sets, int k,
                                          int stride_bytes, kdb_split_mode mode);
KDB_API kdb_status kdb_build_batched_async(void* d_points, const int64_t* h_offsets, int num_sets,
                                           int k, int stride_bytes, kdb_split_mode mode,
                                           void* d_workspace, size_t workspace_bytes,
                                           uint32_t* d_error_word, kdb_stream_t stream);
/* Status of a device error word written by kdb_build_batched_async. */
KDB_API kdb_status kdb_error_word_status(uint32_t word);

/*
 * kdb_build_host -- kdb_build for records in host memory.  Two paths, same
 * output:
 *   - page-locked records that the current device can address (e.g. from
 *     cudaHostAlloc or cudaHostRegister), without payload (stride_bytes = 4k,
 *     k <= 3) and under the default placement: the kernels read the records
 *     and write the tree straight into h_points over the host link; no device
 *     copy of the records is made (every record the build writes is rebuilt
 *     from the 16-byte entry that carries its coordinates);
 *   - otherwise: the records are copied to a device buffer in chunks (of at
 *     least 64 MiB, at most 8) on a stream of the call's own, the build's
 *     first pass over each chunk starting as soon as it has landed, and the
 *     tree is copied back into h_points on `stream`.
 * h_points is written by the device on both paths: page-locked records must
 * not be registered read-only (cudaHostRegisterReadOnly).  On a device error
 * (NaN input, ...) h_points is left as it was.  Synchronises `stream`.
 */
KDB_API kdb_status kdb_build_host(void* h_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                          kdb_stream_t stream);

/*
 * kdb_build_noalloc -- kdb_build that allocates no device memory.
 * The paper has no counterpart; this is a deployment convenience.  Some
 * callers cannot call cudaMalloc (or a stream-ordered allocator) when they
 * build: applications whose whole device-memory budget is fixed and reserved
 * at start-up (for example by another framework's caching allocator), or
 * latency-critical loops where an allocation could fail or stall at an
 * unpredictable moment.  This entry point takes its workspace from one
 * static device array of KDB_NOALLOC_SCRATCH_BYTES compiled into the library;
 * every GPU that loads the library holds that array until the process exits.
 *   d_points, n, k, stride_bytes, mode, stream: as for kdb_build.
 * Limits: n <= KDB_NOALLOC_MAX_POINTS and kdb_workspace_size(n, k,
 * stride_bytes, mode) <= KDB_NOALLOC_SCRATCH_BYTES; anything larger returns
 * KDB_ERR_INVALID_ARGUMENT before any work is enqueued.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * The address is kept for the life of the process, so the library must not
 * be used across a cudaDeviceReset of that device (the reset unloads the
 * array, and the kept address would no longer name it).
 * Every call uses the same array, which keeps the previous call's contents
 * (the build clears what must start at zero): calls that overlap on the GPU,
 * from several streams or host threads, race with each other and must be
 * serialised by the caller.  Synchronises `stream`.
 */
#define KDB_NOALLOC_MAX_POINTS 262144
#define KDB_NOALLOC_SCRATCH_BYTES (64u << 20)
KDB_API kdb_status kdb_build_noalloc(void* d_points, int64_t n, int k, int stride_bytes,
                                     kdb_split_mode mode, kdb_stream_t stream);

/*
 * Steps of the sharded single-tree build.  The paper builds one tree on one
 * GPU; these entry points let several GPUs (one process each) share one tree:
 * the top levels are split across the shards, then each GPU receives the
 * points of one subtree and builds it with kdb_build_subtree.  A shard is
 * d_points[0, n) of the global array, whose original indices are
 * index_base .. index_base + n - 1; the tags (device int32[n], the paper's
 * one int per point, Sec. 3) hold each point's node on the current top
 * level (heap index; the root is 0) or -1 once the point is pinned.  Levels
 * 0 .. 6 (at most 64 nodes).  Each call synchronises `stream` and returns
 * KDB_ERR_INVALID_ARGUMENT for bad arguments, KDB_ERR_INTERNAL if a device
 * check failed (a split dimension >= k, an output position out of range).
 * Keys: a point's key in dimension d is (order-preserving coordinate key <<
 * 32) | original index, so keys are unique and their order is the strict
 * order of Sec. 3.1 with the tie rule.
 *
 * kdb_dist_histogram -- radix-select step of the pivots of level `level`
 * (Observation 1): for every node u of the level (u = tag - (2^level - 1)),
 * count the node's points whose key in dimension d_node_dim[u] agrees with
 * d_node_prefix[u] in its top prefix_bits bits (0, 8, .., 56), by the next 8
 * bits.  d_hist: device uint32[2^level][256], overwritten.
 */
KDB_API kdb_status kdb_dist_histogram(const void* d_points, int64_t n, int k, int stride_bytes,
                                      kdb_split_mode mode, const int32_t* d_tags, int level,
                                      const uint8_t* d_node_dim, const uint64_t* d_node_prefix,
                                      int prefix_bits, uint32_t index_base, uint32_t* d_hist,
                                      kdb_stream_t stream);

/*
 * kdb_dist_box -- smallest and largest coordinate key of every node's points
 * of level `level` in every dimension (the scene box of Sec. 6 at level 0;
 * the tight boxes of the tight-box rule).  d_box: device uint32[2^level][2k]
 * (k minima, then k maxima), overwritten; a node without points on this
 * shard gets 0xFFFFFFFF minima and 0 maxima.
 */
KDB_API kdb_status kdb_dist_box(const void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                                const int32_t* d_tags, int level, uint32_t* d_box, kdb_stream_t stream);

/*
 * kdb_dist_assign -- tag update of level `level` (Sec. 3.2): a point of node
 * t whose key in dimension d_node_dim[u] is below the node's pivot key
 * d_pivot[u] moves to 2t+1, above it to 2t+2; the point equal to it is
 * pinned (tag -1) and its shard position written to d_pinned[u] (device
 * int64[2^level]; entries of nodes whose pivot is elsewhere are untouched).
 */
KDB_API kdb_status kdb_dist_assign(const void* d_points, int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                                   int32_t* d_tags, int level, const uint8_t* d_node_dim,
                                   const uint64_t* d_pivot, uint32_t index_base, int64_t* d_pinned,
                                   kdb_stream_t stream);

/*
 * kdb_dist_partition -- the points whose tag is in [first_node, first_node +
 * num_dest) (num_dest <= 64), grouped by destination j = tag - first_node in
 * their shard order (a stable partition), for the exchange: records to
 * d_out_points (device, at least the selected records), their original
 * indices to d_out_index (device uint32).  h_counts: host int64[num_dest],
 * the records of each destination.  Other points (pinned) are left out.
 */
KDB_API kdb_status kdb_dist_partition(const void* d_points, int64_t n, int stride_bytes, const int32_t* d_tags,
                                      int32_t first_node, int num_dest, uint32_t index_base, void* d_out_points,
                                      uint32_t* d_out_index, int64_t* h_counts, kdb_stream_t stream);

/*
 * Plans: a build prepared once and enqueued many times, for repeated builds
 * of the same shape and for CUDA-graph capture.  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * kdb_plan_create -- plans builds of num_sets sets laid out as for
 * kdb_build_batched (h_offsets: host int64[num_sets+1], h_offsets[0] = 0,
 * non-decreasing; num_sets = 1 and {0, N} for a single tree), with k,
 * stride_bytes and mode as for kdb_build.  Allocates the plan's device
 * workspace (kdb_plan_workspace_bytes) on the current device, copies its
 * tables there, and runs one build on zero-filled points so that every
 * kernel is loaded and configured.  Synchronous.  *out_plan is NULL on error.
 *
 * kdb_plan_enqueue -- enqueues one build of d_points (device, in/out, the
 * planned layout) on `stream` and returns without synchronising.  It
 * allocates nothing, synchronises nothing and reads no host memory: only
 * kernels and memsets on `stream`, so it may be captured into a CUDA graph
 * (in any capture mode) and the graph replayed on new point data.  The
 * current device must be the plan's.  Builds of one plan share its
 * workspace: enqueue them in one stream order.  Returns
 * KDB_ERR_INVALID_ARGUMENT or KDB_ERR_CUDA for launch problems; device
 * errors (NaN, timeouts) are read with kdb_plan_status.  On a device error
 * the records are left as they were (as for kdb_build).
 *
 * kdb_plan_status -- synchronises `stream` and returns the device status of
 * the plan's last build enqueued before that point.
 *
 * kdb_plan_destroy -- frees the plan (NULL is ignored); the caller makes
 * sure no enqueued build of it is still running.
 */
typedef struct kdb_plan_st* kdb_plan;
KDB_API kdb_status kdb_plan_create(const int64_t* h_offsets, int num_sets, int k, int stride_bytes,
                                   kdb_split_mode mode, kdb_plan* out_plan);
KDB_API kdb_status kdb_plan_enqueue(kdb_plan plan, void* d_points, kdb_stream_t stream);
KDB_API kdb_status kdb_plan_status(kdb_plan plan, kdb_stream_t stream);
KDB_API size_t kdb_plan_workspace_bytes(kdb_plan plan);
KDB_API void kdb_plan_destroy(kdb_plan plan);

/*
 * Build server: requests accepted as they arrive and built on one GPU by
 * continuous batching.  The paper has no counterpart; each request is the
 * paper's build (Sec. 3.2) of its own point set, bit-identical to kdb_build
 * of that set alone, whatever it was batched with.
 *
 * A worker thread owns max_inflight_batches CUDA streams.  Whenever one is
 * free, the queued requests with the head request's layout (k, stride_bytes,
 * mode) are taken in arrival order, as many as fit in the free part of the
 * device-memory budget (points plus build workspace) and the caps, and are
 * enqueued as one batch: copies in, one kdb_build_batched_async, copies out.
 * Requests arriving meanwhile go to the next free stream, so batches overlap
 * on the device.  The budget is reserved from the device when the server is
 * created and stays reserved until it is destroyed.  A batch that fails on
 * the device (NaN input, a timeout) leaves the records untouched; each of its
 * requests is then run again alone, so only the failing request fails.
 *
 * kdb_server_create -- on the current device; fails with
 *   KDB_ERR_OUT_OF_MEMORY if budget_bytes exceeds the free device memory.
 * kdb_server_submit -- queues one build.  h_points: host, n records as for
 *   kdb_build (pinned memory gives asynchronous copies; pageable memory
 *   works but serialises the copies); read when the request's batch starts,
 *   so it must stay valid and unchanged until the result is polled.  h_out:
 *   host, n records, receives the tree (may equal h_points; NULL = no copy
 *   back).  *out_id receives the request id.  Returns
 *   KDB_ERR_INVALID_ARGUMENT for bad arguments and KDB_ERR_OUT_OF_MEMORY if
 *   the request alone exceeds the budget; nothing is queued then.
 * kdb_server_poll -- moves up to max_results finished requests into out,
 *   waiting up to timeout_ms (0: no wait, < 0: until one is there) for the
 *   first.  Returns the count (-1 for bad arguments).  Times are seconds
 *   since the server was created: submit, admission into a batch, and the end
 *   of the batch's copy out.
 * kdb_server_get_stats -- counters since creation.
 * kdb_server_destroy -- builds everything still queued, waits for it, frees
 *   the server.  Results not yet polled are dropped.
 * Submit, poll and stats may be called from any thread.
 */
typedef struct kdb_server_st* kdb_server;
typedef struct {
  size_t budget_bytes;         /* device memory for in-flight batches */
  int max_inflight_batches;    /* streams, 1 .. 16 */
  int max_batch_requests;      /* >= 1 */
  int64_t max_batch_points;    /* >= 1; a single larger request still runs */
} kdb_server_config;
typedef struct {
  int64_t id;
  kdb_status status;
  int64_t n;
  double submit_s, admit_s, done_s;
} kdb_request_result;
typedef struct {
  int64_t submitted, completed, failed;
  int64_t batches, retried_alone;
  int64_t max_batch_requests, max_inflight_batches;
  int64_t queued, inflight_requests;
  size_t budget_bytes, used_bytes, max_used_bytes;
} kdb_server_stats;
KDB_API kdb_status kdb_server_create(const kdb_server_config* config, kdb_server* out_server);
KDB_API kdb_status kdb_server_submit(kdb_server server, const void* h_points, void* h_out, int64_t n,
                                     int k, int stride_bytes, kdb_split_mode mode, int64_t* out_id);
KDB_API int kdb_server_poll(kdb_server server, kdb_request_result* out, int max_results,
                            int timeout_ms);
KDB_API kdb_status kdb_server_get_stats(kdb_server server, kdb_server_stats* out);
KDB_API kdb_status kdb_server_destroy(kdb_server server);

/*
 * kdb_set_placement -- how the final placement moves the records into level
 * order (Sec. 3.2, 7.1).  Both settings give identical output.
 *   KDB_PLACEMENT_AUTO      (default) when the part of the build's workspace
 *                           that is no longer needed at that point can hold
 *                           the N records, gather them there in node order
 *                           and copy them back (two coalesced passes);
 *                           otherwise as KDB_PLACEMENT_IN_PLACE.
 *   KDB_PLACEMENT_IN_PLACE  the almost-in-place permutation: cycles of the
 *                           node -> original-index array (one int32 per
 *                           point) are walked from one leader per 16 nodes,
 *                           whose records wait in a staging area of N/16
 *                           records.
 * Process-wide; read when a build is enqueued.  Returns the previous setting;
 * any other value leaves the setting unchanged.
 */
typedef enum { KDB_PLACEMENT_AUTO = 0, KDB_PLACEMENT_IN_PLACE = 1 } kdb_placement;
KDB_API kdb_placement kdb_set_placement(kdb_placement placement);

/*
 * kdb_set_memory_mode -- how kdb_build and kdb_build_ex (without caller
 * workspace and without the original-index or split-dimension outputs) size
 * their device memory.  The paper builds with one int per point beside the
 * records (abstract, Sec. 1, Sec. 7.1); the default pipeline trades that for
 * bandwidth (per-dimension lists, kdb_workspace_size).
 *   KDB_MEMORY_AUTO  the default pipeline, unless its workspace does not fit
 *                    the device memory free at the call (plus what the
 *                    library's memory pool holds unused, less 256 MiB): then
 *                    the lean build.
 *   KDB_MEMORY_FAST  always the default pipeline.
 *   KDB_MEMORY_LEAN  always the lean build (N >= 4; smaller N build as usual).
 * The lean build follows the steps of the sharded build with every shard on
 * this GPU: the top 4 levels by a radix select of every node's pivot
 * (Observation 1) over the whole array, one stable move of every point to
 * its level-4 subtree's slice, then each of the 16 subtrees built alone by
 * the default pipeline in a workspace sized for one subtree.  Its device
 * memory (kdb_lean_workspace_size) is one tag and one index per point, a
 * copy of the records, and one subtree's workspace: about 29 B per point for
 * float3 records without payload, against about 146 B for the default.  The
 * output is the same tree.  The records are only read until every subtree is
 * built, so a device error leaves them untouched, as for the default.
 * Synchronous, like kdb_build.  Process-wide; returns the previous setting;
 * any other value leaves it unchanged.
 * kdb_lean_workspace_size -- device bytes the lean build allocates for these
 *   arguments, 0 for invalid arguments or N < 4.
 */
typedef enum { KDB_MEMORY_AUTO = 0, KDB_MEMORY_FAST = 1, KDB_MEMORY_LEAN = 2 } kdb_memory_mode;
KDB_API kdb_memory_mode kdb_set_memory_mode(kdb_memory_mode mode);
KDB_API size_t kdb_lean_workspace_size(int64_t n, int k, int stride_bytes, kdb_split_mode mode);

/*
 * Tuning of the per-dimension-list path (k <= 3).  Three choices, none of
 * which changes the output (every choice gives bit-identical trees):
 *   KDB_TUNE_PARTITION  tile shape of the per-level stable split (the sorts
 *                       of Sec. 3.1 that follow level 0, Observation 1 fused
 *                       in);
 *   KDB_TUNE_RADIX      tile shape of the passes of the level-0 sort;
 *   KDB_TUNE_DIGITS     digit width of the level-0 sort (the radix-key sort
 *                       of Sec. 7.1): a 32-bit key takes 32 / width passes,
 *                       rounded up.
 * The library carries a few compiled shapes and widths.  A shape is threads
 * per block, entries per thread and resident blocks per SM.
 *
 * kdb_tuning_shape_count -- number of shapes (widths for KDB_TUNE_DIGITS) of
 *   `kernel`, or -1 for an unknown kernel.
 * kdb_tuning_shape       -- shape `index` of `kernel` (host out-pointers, each
 *   may be NULL); for KDB_TUNE_DIGITS `threads` receives the width in bits,
 *   `items_per_thread` the passes per key and `blocks_per_sm` 1.
 *   KDB_ERR_INVALID_ARGUMENT for an unknown kernel or index.
 * kdb_get_tuning / kdb_set_tuning -- the process-wide setting.  Default
 *   {0, 0, 8}.  kdb_set_tuning returns KDB_ERR_INVALID_ARGUMENT and changes
 *   nothing if a shape index is out of range or the width is not compiled.
 *
 * The tuning table keeps one setting per kind of build: (bit length of the
 * total point count, k, stride_bytes, mode argument as given).  Every build
 * takes its kind's entry when the table has one, else the process-wide
 * setting, at the time it is planned (kdb_build and friends: at the call;
 * kdb_plan_create: at creation, and a captured graph keeps what it was
 * captured with).  The table holds at most 256 kinds; a new kind beyond
 * that drops the oldest.  Thread safe.
 * kdb_lookup_tuning -- the setting a build of this kind would take; host
 *   out-pointers; *from_table (may be NULL) = 1 if it comes from the table.
 *   KDB_ERR_INVALID_ARGUMENT if `out` is NULL or n < 0.
 * kdb_clear_tuning_table -- forget every kept kind.
 * kdb_autotune -- times every (partition shape, radix shape, width) on the
 *   caller's points, keeps the fastest as the process-wide setting and as
 *   the table entry of this kind of build.
 *     d_points    device, in: n points as for kdb_build; read only (each
 *                 trial builds a copy).
 *     reps        timed builds per choice, 1..64; a choice's time is the
 *                 median.
 *     out_best    host, out (may be NULL): the chosen setting.
 *     out_best_ms host, out (may be NULL): its median build time.
 *     h_ms        host, out (may be NULL): count(PARTITION) x count(RADIX) x
 *                 count(DIGITS) medians, partition shape major, width minor;
 *                 -1 where not timed.  Where the build does not use the
 *                 tuned kernels (k > 3, or n too small for a global level)
 *                 only the current setting is timed and kept, and the table
 *                 is left alone.
 *   Allocates a copy of the points and a workspace from the device's memory
 *   pool and frees them before returning.  Synchronous.  Returns the first
 *   build error, KDB_ERR_OUT_OF_MEMORY, or KDB_ERR_INVALID_ARGUMENT for bad
 *   arguments (as kdb_build, plus n < 2 or reps out of range).
 * The workspace size of a build does not depend on the setting.
 */
enum { KDB_TUNE_PARTITION = 0, KDB_TUNE_RADIX = 1, KDB_TUNE_DIGITS = 2 };
typedef struct {
  int32_t partition_shape;  /* index into the partition shapes */
  int32_t radix_shape;      /* index into the radix shapes */
  int32_t digit_bits;       /* level-0 digit width in bits (a compiled width) */
} kdb_tuning;
KDB_API int kdb_tuning_shape_count(int kernel);
KDB_API kdb_status kdb_tuning_shape(int kernel, int index, int* threads, int* items_per_thread,
                                    int* blocks_per_sm);
KDB_API kdb_status kdb_get_tuning(kdb_tuning* out);
KDB_API kdb_status kdb_set_tuning(const kdb_tuning* tuning);
KDB_API kdb_status kdb_lookup_tuning(int64_t n, int k, int stride_bytes, kdb_split_mode mode,
                                     kdb_tuning* out, int* from_table);
KDB_API void kdb_clear_tuning_table(void);
KDB_API kdb_status kdb_autotune(const void* d_points, int64_t n, int k, int stride_bytes,
                                kdb_split_mode mode, int reps, kdb_tuning* out_best,
                                float* out_best_ms, float* h_ms, kdb_stream_t stream);
/*
 * kdb_save_tuning / kdb_load_tuning -- the process-wide setting and the table
 * as a small JSON file:
 *   {"partition": [threads, items, blocks], "radix": [threads, items, blocks],
 *    "digit_bits": w, "table": [{"log2n": b, "k": k, "stride": s, "mode": m,
 *    "partition": [...], "radix": [...], "digit_bits": w}, ...]}
 * Shapes are stored by value, so a file from a library with other compiled
 * shapes or widths is refused on load (KDB_ERR_INVALID_ARGUMENT, setting and
 * table unchanged), as are unreadable or malformed files and tables of more
 * than 256 entries.  A missing "digit_bits" reads as 8 and a missing "table"
 * as an empty one; loading replaces the setting and the whole table.  Saving
 * returns KDB_ERR_INVALID_ARGUMENT if the file cannot be written.  Host only.
 */
KDB_API kdb_status kdb_save_tuning(const char* path);
KDB_API kdb_status kdb_load_tuning(const char* path);

/*
 * kdb_validate -- check the k-d condition of a level-order tree (Sec. 1):
 * for every node i and every ancestor p with split dimension d, x_d(i) <=
 * x_d(p) if i is in p's left subtree and >= if in the right one, under the
 * total order with -0.0 < +0.0.  For the widest mode the dimensions are
 * recomputed top-down from the tree's own planes (Sec. 6).
 *   h_first_bad_node  host, out: smallest violating node, or -1.
 * Returns KDB_OK or KDB_ERR_NOT_A_KD_TREE.  Synchronous.
 */
KDB_API kdb_status kdb_validate(const void* d_points, int64_t n, int k, int stride_bytes,
                        kdb_split_mode mode, int64_t* h_first_bad_node, kdb_stream_t stream);

/*
 * Profiling of the library's own kernels (tracing for benchmarks).
 * kdb_profile_start() makes every later build record a CUDA event pair around
 * each of its kernel launches, on the launch stream; kdb_profile_stop()
 * waits for those events and fills up to max_entries rows, one per kernel
 * kind, with the number of launches, their summed device time and their
 * summed algorithmic bytes (the bytes the kernel's job has to read and write,
 * not measured traffic).  Returns the number of rows, or -1 on a CUDA error.
 * kdb_launch_count() is the number of kernels the library has launched in
 * this process.  Host-side state shared by all threads; for benchmarks.
 */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double bytes;
} kdb_kernel_stat;
KDB_API void kdb_profile_start(void);
KDB_API int kdb_profile_stop(kdb_kernel_stat* out, int max_entries);
KDB_API int64_t kdb_launch_count(void);

/*
 * Fault injection for tests (host-side; never faults a GPU):
 *   KDB_FAULT_ALLOC       the next workspace allocation reports failure;
 *   KDB_FAULT_LOOKBACK    the next build's radix passes wait on a status value
 *                         that no block ever writes, so each bounded wait runs
 *                         out after about `arg` microseconds and the build
 *                         returns KDB_ERR_TIMEOUT.
 *   KDB_FAULT_LOOKBACK_PARTITION  the same for the next build's per-level
 *                         partition passes only, which run after the first
 *                         pivots have been placed.
 *   KDB_FAULT_LOW_MEMORY  the next automatic memory-mode decision
 *                         (kdb_set_memory_mode) sees only `arg` bytes free.
 * Returns the previous fault setting.  Not thread-safe; tests only.
 */
enum {
  KDB_FAULT_NONE = 0,
  KDB_FAULT_ALLOC = 1,
  KDB_FAULT_LOOKBACK = 2,
  KDB_FAULT_LOOKBACK_PARTITION = 3,
  KDB_FAULT_LOW_MEMORY = 4
};
KDB_API int kdb_debug_inject_fault(int fault, int64_t arg);

#ifdef __cplusplus
}
#endif

#endif /* KDB_H */
