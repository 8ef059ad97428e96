/*
 * paper_cpu.c -- the paper's level loop on host threads: a parallel CPU
 * baseline for the benchmark, NOT the oracle.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the rest of this directory:
 * nothing on the product path calls, links or loads it, and it shares no code
 * with the CUDA library.  The tests check it against the recursive oracle in
 * kd_oracle.c.
 *
 * Wald's build (arXiv 2211.00120) is written for GPUs but, as its Sec. 7.2
 * notes, it needs only a parallel sort and a parallel loop, so it ports to
 * any parallel CPU framework.  This is that port, with POSIX threads:
 *
 *   tags = 0 (Sec. 3)
 *   for l = 0 .. L-2:
 *     sort the (tag, point) pairs by less(): tag, then the coordinate in the
 *       tag's split dimension, then (tie rule) the original index (Sec. 3.1);
 *       the prefix [0, F(l-1)) is already final and is skipped (Sec. 7.1);
 *     update every tag from its array position with the O(1) subtree size ss
 *       and segment begin sb (Sec. 3.2, 4.1, 4.2): left of the pivot ->
 *       lChild, right of it -> rChild, the pivot itself stays (pinned);
 *     split dimension of every new subtree (Sec. 6): the scene box clipped by
 *       the new plane and every ancestor's plane; or, for the tight-box rule,
 *       the box of the subtree's points (which form one contiguous run);
 *   final "sort" by tag: the tags are the nodes, so it is a scatter.
 *
 * The sort uses the structure the paper points out (Obs. 2 and 3): after an
 * update the points of each new subtree form one contiguous run (left of
 * their parent's pivot, or right of it), and the parents' pivots sit between
 * the runs.  Sorting by (tag, coordinate, index) therefore moves each pivot
 * to its node's slot in the prefix, moves each run to its segment begin sb,
 * and sorts each run by (coordinate, index).  The moves are one parallel
 * pass; the runs are sorted in parallel, and a run larger than one thread's
 * share by a parallel merge sort.  Coordinates are compared as
 * order-preserving 32-bit keys (float32 with -0 < +0, int32 or uint32).
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum { PC_OK = 0, PC_INVALID = 1, PC_NOMEM = 2, PC_NAN = 4 };
enum { PC_RR = 0, PC_WIDEST = 1, PC_TIGHT = 2, PC_INT32 = 0x100, PC_UINT32 = 0x200 };
#define PC_MAXK 8
#define PC_MAXT 256

typedef struct {
  uint32_t tag; /* subtree id (node of the level-l subtree the point is in) */
  uint32_t idx; /* original index */
} item;

typedef struct {
  const uint32_t* keys; /* k arrays of N keys */
  int64_t N;
  int k, mode, ints;
  const uint8_t* dims; /* split dimension per node (widest / tight) */
  int level;
} ctx_t;

/* ints: 0 float32, 1 int32 (sign bit flipped), 2 uint32 (the bits) */
static uint32_t key_of_bits(uint32_t b, int ints) {
  if (ints == 2) return b;
  if (ints) return b ^ 0x80000000u;
  return b ^ ((b & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u);
}
static float float_of_key(uint32_t key) {
  uint32_t b = key ^ ((key & 0x80000000u) ? 0x80000000u : 0xFFFFFFFFu);
  float f;
  memcpy(&f, &b, 4);
  return f;
}

static int dim_of(const ctx_t* C, uint32_t tag) {
  return C->mode == PC_RR ? C->level % C->k : C->dims[tag];
}

/* Within one run every point carries the same tag, so less() of Sec. 3.1
 * with the tie rule is the order of (key in the run's dimension, original
 * index), packed into one 64-bit value: runs are sorted as integers. */

/* ------------------------------------------------------------ merge sort -- */
static void merge_runs(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, uint64_t* out) {
  int64_t i = 0, j = 0, o = 0;
  while (i < na && j < nb) out[o++] = b[j] < a[i] ? b[j++] : a[i++];
  while (i < na) out[o++] = a[i++];
  while (j < nb) out[o++] = b[j++];
}

static void seq_sort(uint64_t* a, uint64_t* tmp, int64_t n) {
  if (n < 2) return;
  if (n <= 16) { /* insertion sort */
    for (int64_t i = 1; i < n; ++i) {
      uint64_t x = a[i];
      int64_t j = i;
      while (j > 0 && x < a[j - 1]) {
        a[j] = a[j - 1];
        --j;
      }
      a[j] = x;
    }
    return;
  }
  int64_t h = n / 2;
  seq_sort(a, tmp, h);
  seq_sort(a + h, tmp + h, n - h);
  merge_runs(a, h, a + h, n - h, tmp);
  memcpy(a, tmp, (size_t)n * sizeof *a);
}

/* Split of a merge of a[0..na) and b[0..nb) at output position p: the number
 * of elements taken from a (merge path; values are distinct). */
static int64_t merge_split(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, int64_t p) {
  int64_t lo = p > nb ? p - nb : 0, hi = p < na ? p : na;
  while (lo < hi) {
    int64_t i = (lo + hi) / 2, j = p - i - 1;
    if (j >= 0 && j < nb && b[j] < a[i]) hi = i;
    else lo = i + 1;
  }
  return lo;
}

typedef struct {
  uint64_t *src, *dst;
  int64_t n;
  int t, T, w; /* thread, threads, run width of this round (in chunks) */
} psort_arg;

static void run_threads(void* (*fn)(void*), void* args, size_t sz, int T);

/* Round 0: thread t sorts its chunk of src in place. */
static void* psort_chunk(void* p) {
  psort_arg* A = (psort_arg*)p;
  int64_t b0 = A->n * A->t / A->T, b1 = A->n * (A->t + 1) / A->T;
  seq_sort(A->src + b0, A->dst + b0, b1 - b0);
  return NULL;
}

/* Round w: runs of w chunks are merged pairwise from src into dst; each merge
 * is split over the threads that own its chunks, by merge path. */
static void* psort_merge(void* p) {
  psort_arg* A = (psort_arg*)p;
  const int T = A->T, t = A->t, w = A->w;
  const int64_t n = A->n;
  int first = t / (2 * w) * 2 * w, mid = first + w, last = first + 2 * w;
  if (mid > T) mid = T;
  if (last > T) last = T;
  int64_t s0 = n * first / T, s1 = n * mid / T, s2 = n * last / T;
  int64_t na = s1 - s0, nb = s2 - s1, tot = na + nb;
  int part = t - first, parts = last - first;
  int64_t p0 = tot * part / parts, p1 = tot * (part + 1) / parts;
  int64_t i0 = merge_split(A->src + s0, na, A->src + s1, nb, p0);
  int64_t i1 = merge_split(A->src + s0, na, A->src + s1, nb, p1);
  merge_runs(A->src + s0 + i0, i1 - i0, A->src + s1 + (p0 - i0), (p1 - i1) - (p0 - i0),
             A->dst + s0 + p0);
  return NULL;
}

/* Sorts a[0..n) with T threads (fork and join per round, no barriers). */
static void parallel_sort(uint64_t* a, uint64_t* tmp, int64_t n, int T) {
  if (T <= 1 || n < 4096) {
    seq_sort(a, tmp, n);
    return;
  }
  psort_arg args[PC_MAXT];
  for (int t = 0; t < T; ++t) args[t] = (psort_arg){a, tmp, n, t, T, 0};
  run_threads(psort_chunk, args, sizeof args[0], T);
  uint64_t *src = a, *dst = tmp;
  for (int w = 1; w < T; w *= 2) {
    for (int t = 0; t < T; ++t) args[t] = (psort_arg){src, dst, n, t, T, w};
    run_threads(psort_merge, args, sizeof args[0], T);
    uint64_t* x = src;
    src = dst;
    dst = x;
  }
  if (src != a) memcpy(a, src, (size_t)n * sizeof *a);
}

/* ------------------------------------------------- O(1) ss and sb (Sec. 4) */
static int num_levels(int64_t n) {
  int L = 0;
  while (n >> L) ++L;
  return L;
}
static int level_of(uint32_t s) { return num_levels((int64_t)s + 1) - 1; }
static int64_t full_nodes(int l) { return l < 0 ? 0 : (((int64_t)1 << l) - 1); }

/* ss(s): nodes in the subtree of s (Sec. 4.1) */
static int64_t ss(int64_t s, int64_t N) {
  if (s >= N) return 0;
  int L = num_levels(N), h = L - level_of((uint32_t)s) - 1;
  int64_t fllc = ((s + 1) << h) - 1; /* first lowest-level child */
  int64_t low = N - fllc;
  if (low < 0) low = 0;
  if (low > ((int64_t)1 << h)) low = (int64_t)1 << h;
  return (((int64_t)1 << h) - 1) + low;
}
/* sb(s, l): first position of subtree s's segment after the level-l sort (Sec. 4.2) */
static int64_t sb(int64_t s, int l, int64_t N) {
  int L = num_levels(N), h = L - l - 1;
  int64_t nls = s - full_nodes(l); /* left siblings on level l */
  int64_t low = nls << h, m = N - full_nodes(L - 1);
  if (low > m) low = m;
  return full_nodes(l) + nls * (((int64_t)1 << h) - 1) + low;
}

/* ------------------------------------------------------------ the build -- */
typedef struct {
  ctx_t* C;
  item* a;
  uint64_t *v, *vt; /* packed values and merge scratch, N each */
  int64_t N;
  int l, t, T;
  int64_t seg_lo, seg_hi; /* subtrees of level l handled by this thread */
} lvl_arg;

/* Run [b, b + n) of subtree s: pack (key in s's dimension, index). */
static void pack_run(const ctx_t* C, const item* a, uint64_t* v, int64_t b, int64_t n, uint32_t s) {
  const uint32_t* kd = C->keys + (int64_t)dim_of(C, s) * C->N;
  for (int64_t i = b; i < b + n; ++i) v[i] = ((uint64_t)kd[a[i].idx] << 32) | a[i].idx;
}
static void unpack_run(item* a, const uint64_t* v, int64_t b, int64_t n) {
  for (int64_t i = b; i < b + n; ++i) a[i].idx = (uint32_t)v[i];
}

/* Sort the runs of subtrees [seg_lo, seg_hi) of level l, each by itself. */
static void* sort_segments(void* p) {
  lvl_arg* A = (lvl_arg*)p;
  for (int64_t s = A->seg_lo; s < A->seg_hi; ++s) {
    int64_t b = sb(s, A->l, A->N), n = ss(s, A->N);
    if (n < 2) continue;
    pack_run(A->C, A->a, A->v, b, n, (uint32_t)s);
    seq_sort(A->v + b, A->vt + b, n);
    unpack_run(A->a, A->v, b, n);
  }
  return NULL;
}

typedef struct {
  ctx_t* C;
  item* a;
  int64_t N, lo, hi;
  int l;
  item* out;
} upd_arg;

/* The moves of the level-l sort for positions [lo, hi) of the array as the
 * level l-1 update left it: a pivot of level l-1 (its tag is still its node,
 * below F(l)) goes to slot tag; any other point is in the run of its new
 * subtree c, which starts at the parent's segment begin (left child) or just
 * after the parent's pivot (right child), and keeps its place in that run. */
static void* move_to_segments(void* p) {
  upd_arg* A = (upd_arg*)p;
  const int l = A->l;
  for (int64_t i = A->lo; i < A->hi; ++i) {
    item it = A->a[i];
    int64_t c = it.tag;
    if (c < full_nodes(l)) {
      A->out[c] = it;
      continue;
    }
    int64_t par = (c - 1) / 2;
    int64_t start = sb(par, l - 1, A->N);
    if (c == 2 * par + 2) start += ss(2 * par + 1, A->N) + 1;
    A->out[sb(c, l, A->N) + (i - start)] = it;
  }
  return NULL;
}

/* Tag update of Sec. 3.2 for positions [lo, hi). */
static void* update_tags(void* p) {
  upd_arg* A = (upd_arg*)p;
  for (int64_t i = A->lo; i < A->hi; ++i) {
    int64_t s = A->a[i].tag;
    int64_t pivot = sb(s, A->l, A->N) + ss(2 * s + 1, A->N);
    if (i < pivot) A->a[i].tag = (uint32_t)(2 * s + 1);
    else if (i > pivot) A->a[i].tag = (uint32_t)(2 * s + 2);
  }
  return NULL;
}

static void run_threads(void* (*fn)(void*), void* args, size_t sz, int T) {
  pthread_t th[PC_MAXT];
  int started[PC_MAXT] = {0};
  for (int t = 1; t < T; ++t)
    started[t] = pthread_create(&th[t], NULL, fn, (char*)args + sz * t) == 0;
  fn(args);
  for (int t = 1; t < T; ++t) {
    if (started[t]) pthread_join(th[t], NULL);
    else fn((char*)args + sz * t); /* could not start a thread: do its part here */
  }
}

static int widest_keys(const uint32_t* lo, const uint32_t* hi, int k, int ints) {
  int best = 0;
  if (ints) {
    /* both integer key maps keep differences: the extent is the key range */
    int64_t be = 0;
    for (int d = 0; d < k; ++d) {
      int64_t e = (int64_t)hi[d] - (int64_t)lo[d];
      if (d == 0 || e > be) { be = e; best = d; }
    }
    return best;
  }
  float be = 0.0f;
  for (int d = 0; d < k; ++d) {
    float e = float_of_key(hi[d]) - float_of_key(lo[d]);
    if (d == 0 || e > be) { be = e; best = d; }
  }
  return best;
}

int pc_build(const void* points, int64_t N, int k, int stride, int mode, int threads,
             int32_t* out_orig) {
  if (N < 0 || N > 2147483647LL || k < 1 || k > PC_MAXK || stride < 4 * k || stride % 4) return PC_INVALID;
  if ((mode & PC_INT32) && (mode & PC_UINT32)) return PC_INVALID;
  const int ints = (mode & PC_INT32) ? 1 : ((mode & PC_UINT32) ? 2 : 0);
  mode &= 0xFF;
  if (mode != PC_RR && mode != PC_WIDEST && mode != PC_TIGHT) return PC_INVALID;
  if (ints && mode == PC_WIDEST) return PC_INVALID;
  if (N == 0) return PC_OK;
  if (!points || !out_orig) return PC_INVALID;
  int T = threads > 0 ? threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (T < 1) T = 1;
  if (T > PC_MAXT) T = PC_MAXT;
  const unsigned char* base = (const unsigned char*)points;
  uint32_t* keys = (uint32_t*)malloc((size_t)N * k * sizeof *keys);
  item* a = (item*)malloc((size_t)N * sizeof *a);
  item* tmp = (item*)malloc((size_t)N * sizeof *tmp);
  uint64_t* v = (uint64_t*)malloc((size_t)N * sizeof *v);
  uint64_t* vt = (uint64_t*)malloc((size_t)N * sizeof *vt);
  uint8_t* dims = (uint8_t*)calloc((size_t)N, 1);
  float* lo = (float*)malloc((size_t)N * k * sizeof(float)); /* clipped domain per node */
  float* hi = (float*)malloc((size_t)N * k * sizeof(float));
  if (!keys || !a || !tmp || !v || !vt || !dims || !lo || !hi) {
    free(keys); free(a); free(tmp); free(v); free(vt); free(dims); free(lo); free(hi);
    return PC_NOMEM;
  }
  int rc = PC_OK;
  uint32_t blo[PC_MAXK], bhi[PC_MAXK];
  for (int d = 0; d < k; ++d) {
    blo[d] = 0xFFFFFFFFu;
    bhi[d] = 0;
  }
  for (int64_t i = 0; i < N && rc == PC_OK; ++i) {
    for (int d = 0; d < k; ++d) {
      uint32_t b;
      memcpy(&b, base + i * stride + 4 * d, 4);
      if (!ints && (b & 0x7FFFFFFFu) > 0x7F800000u) rc = PC_NAN;
      uint32_t key = key_of_bits(b, ints);
      keys[(int64_t)d * N + i] = key;
      if (key < blo[d]) blo[d] = key;
      if (key > bhi[d]) bhi[d] = key;
    }
    a[i].tag = 0;
    a[i].idx = (uint32_t)i;
  }
  ctx_t C = {keys, N, k, mode, ints, dims, 0};
  if (rc == PC_OK && mode != PC_RR) {
    /* the scene box: the root's domain and its tight box (Sec. 6) */
    dims[0] = (uint8_t)widest_keys(blo, bhi, k, ints);
    for (int d = 0; d < k; ++d) {
      lo[d] = float_of_key(blo[d]);
      hi[d] = float_of_key(bhi[d]);
    }
  }
  const int L = num_levels(N);
  lvl_arg la[PC_MAXT];
  upd_arg ua[PC_MAXT];
  for (int l = 0; l + 1 < L && rc == PC_OK; ++l) {
    C.level = l;
    /* sort by less(): pivots of level l-1 to their slots, every subtree of
       level l (one contiguous run after the previous update, Obs. 3) to its
       segment, then each run sorted by itself */
    const int64_t nseg = (int64_t)1 << l;
    const int64_t live = N - full_nodes(l);
    if (l > 0) {
      const int64_t b0 = full_nodes(l - 1), n0 = N - b0;
      for (int t = 0; t < T; ++t)
        ua[t] = (upd_arg){&C, a, N, b0 + n0 * t / T, b0 + n0 * (t + 1) / T, l, tmp};
      run_threads(move_to_segments, ua, sizeof ua[0], T);
      memcpy(a + b0, tmp + b0, (size_t)n0 * sizeof *a);
    }
    if (nseg < T && live > 4096) {
      for (int64_t s = full_nodes(l); s < full_nodes(l) + nseg; ++s) {
        int64_t b = sb(s, l, N), n = ss(s, N);
        if (n < 2) continue;
        pack_run(&C, a, v, b, n, (uint32_t)s);
        parallel_sort(v + b, vt + b, n, T);
        unpack_run(a, v, b, n);
      }
    } else {
      for (int t = 0; t < T; ++t)
        la[t] = (lvl_arg){&C, a, v, vt, N, l, t, T, full_nodes(l) + nseg * t / T,
                          full_nodes(l) + nseg * (t + 1) / T};
      run_threads(sort_segments, la, sizeof la[0], T);
    }
    if (rc != PC_OK) break;
    /* tag update over the live positions [F(l), N) */
    for (int t = 0; t < T; ++t) {
      int64_t b = full_nodes(l);
      ua[t] = (upd_arg){&C, a, N, b + live * t / T, b + live * (t + 1) / T, l, NULL};
    }
    run_threads(update_tags, ua, sizeof ua[0], T);
    /* split dimensions of the new subtrees of level l + 1 */
    if (mode != PC_RR) {
      for (int64_t s = full_nodes(l); s < full_nodes(l + 1) && s < N; ++s) {
        int64_t b = sb(s, l, N), piv = b + ss(2 * s + 1, N), e = b + ss(s, N);
        int ds = dims[s];
        for (int side = 0; side < 2; ++side) {
          int64_t c = 2 * s + 1 + side;
          if (c >= N) break;
          int64_t r0 = side ? piv + 1 : b, r1 = side ? e : piv; /* the child's run */
          if (mode == PC_TIGHT) {
            uint32_t tl[PC_MAXK], th2[PC_MAXK];
            for (int d = 0; d < k; ++d) {
              tl[d] = 0xFFFFFFFFu;
              th2[d] = 0;
            }
            for (int64_t i = r0; i < r1; ++i)
              for (int d = 0; d < k; ++d) {
                uint32_t key = keys[(int64_t)d * N + a[i].idx];
                if (key < tl[d]) tl[d] = key;
                if (key > th2[d]) th2[d] = key;
              }
            dims[c] = (uint8_t)widest_keys(tl, th2, k, ints);
          } else {
            /* the parent's domain clipped by the parent's plane (the pivot) */
            float* cl = lo + c * k;
            float* ch = hi + c * k;
            memcpy(cl, lo + s * k, sizeof(float) * k);
            memcpy(ch, hi + s * k, sizeof(float) * k);
            float x = float_of_key(keys[(int64_t)ds * N + a[piv].idx]);
            if (side == 0) ch[ds] = x; else cl[ds] = x;
            float be = 0.0f;
            int best = 0;
            for (int d = 0; d < k; ++d) {
              float ext = ch[d] - cl[d];
              if (d == 0 || ext > be) { be = ext; best = d; }
            }
            dims[c] = (uint8_t)best;
          }
        }
      }
    }
  }
  if (rc == PC_OK) /* final "sort" by tag: every tag is now its node */
    for (int64_t i = 0; i < N; ++i) out_orig[a[i].tag] = (int32_t)a[i].idx;
  free(keys); free(a); free(tmp); free(v); free(vt); free(dims); free(lo); free(hi);
  return rc;
}
