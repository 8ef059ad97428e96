/*
 * kd_oracle.c -- CPU oracle for the left-balanced, complete k-d tree build.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (Wald, "GPU-friendly, Parallel, and (Almost-)In-Place
 * Construction of Left-Balanced k-d Trees", arXiv 2211.00120):
 *
 *   The tree is stored in level order, node i at array slot i, children of i
 *   at 2i+1 and 2i+2 (Sec. 2).  It is left-balanced and complete: every level
 *   but the last is full and the last is filled from the left (Sec. 4.1).
 *   Every node must be >= all nodes of its left subtree and <= all nodes of
 *   its right subtree in its split dimension (Sec. 1).  The split dimension is
 *   level mod k for round robin (Sec. 2) or, for the split-widest extension,
 *   the dimension in which the subtree's domain is widest, the domain being
 *   the scene bounding box clipped by every ancestor's plane (Sec. 6).  A
 *   third mode, which the paper does not have, takes the widest side of the
 *   subtree's tight bounding box instead (the box of the subtree's own
 *   points, not its domain); it gives other trees than Sec. 6.
 *
 *   Observation 1 (Sec. 2.1) says that once a subtree's points are sorted in
 *   its split dimension, the point at rank ss(lChild(s)) is node s, lower
 *   ranks form the left subtree and higher ranks the right one.  This oracle
 *   is that definition run recursively ("sort, split, recurse", the usual
 *   list-based builder the paper contrasts itself with in Sec. 1), NOT the
 *   paper's tag/sort level loop.
 *
 * Readings of points the paper leaves open:
 *   - ties: points are ordered by (coordinate, original index), so the valid
 *     tree is unique; -0.0 orders before +0.0 (the paper compares with '<'
 *     and is silent on equal keys);
 *   - NaN coordinates are rejected (KDO_NAN);
 *   - coordinates are float32 unless the mode argument carries KDO_INT32
 *     (the paper's int1 / int2 data, Table 1 and Sec. 5) or KDO_UINT32
 *     (another scalar type of the templated builder, Sec. 7.2): then they
 *     are int32 or uint32, ordered as signed or unsigned integers, and box
 *     extents are exact 64-bit differences.  The clipped-domain rule is
 *     float-only here (its planes clip a float box); an integer type with it,
 *     or both flags at once, is refused as an invalid argument;
 *   - the widest dimension is argmax over d of (hi[d] - lo[d]) computed in
 *     float32, scanned from d = 0 with a strict '>', so the lowest dimension
 *     wins ties; box corners are the smallest and largest coordinate under
 *     the strict order (-0.0 below +0.0);
 *   - subtree sizes are counted level by level here, not with the paper's
 *     O(1) formula (Sec. 4.1), so that the two can be checked against each
 *     other.
 *
 * Parity pins (see tests/test_oracle_pins.py): the 6-point set of Fig. 1, the
 * final array of the 10-point walkthrough of Sec. 5, brute force over all N!
 * arrangements for N <= 7, the k = 1 case against the textbook level-order
 * (Eytzinger) layout of a sorted array, k-d and permutation invariants, and
 * agreement with a separate step-by-step emulator of the paper's level loop;
 * for integer coordinates also the walkthrough as int2 points, values on both
 * sides of 2^31 (a signed/unsigned mix-up fails the k = 1 pin), and the
 * uint32 tree of any values equal to the int32 tree of the same values with
 * the top bit flipped.  The subtree entry (kdo_build_sub) is pinned by the
 * whole build: rebuilt on their own, the subtrees of a whole build are the
 * same subtrees, and round robin started at dimension f is the build of the
 * coordinates rotated by f.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { KDO_OK = 0, KDO_INVALID = 1, KDO_NOMEM = 2, KDO_NAN = 4, KDO_NOT_KD = 6 };
enum { KDO_ROUND_ROBIN = 0, KDO_WIDEST = 1, KDO_WIDEST_TIGHT = 2 };
/* flags in the mode argument: int32 or uint32 coordinates */
enum { KDO_INT32 = 0x100, KDO_UINT32 = 0x200 };
#define KDO_MAXK 8

typedef struct {
  const unsigned char* base; /* first record */
  int64_t stride;            /* bytes between records */
  int k;                     /* coordinates per record (4-byte items at offsets 0,4,..) */
  int ints;                  /* 0: float32, 1: int32, 2: uint32 coordinates */
} pointset;

static float coord(const pointset* P, int64_t i, int d) {
  float v;
  memcpy(&v, P->base + i * P->stride + 4 * (int64_t)d, sizeof v);
  return v;
}

/* An integer coordinate as a 64-bit value: int32 or uint32 by the type. */
static int64_t icoord(const pointset* P, int64_t i, int d) {
  if (P->ints == 2) {
    uint32_t u;
    memcpy(&u, P->base + i * P->stride + 4 * (int64_t)d, sizeof u);
    return (int64_t)u;
  }
  int32_t v;
  memcpy(&v, P->base + i * P->stride + 4 * (int64_t)d, sizeof v);
  return (int64_t)v;
}

static int coord_type(int mode) {
  return (mode & KDO_INT32) ? 1 : ((mode & KDO_UINT32) ? 2 : 0);
}

/* Strict total order on (value, original index); -0.0 < +0.0.  Returns <0,
 * 0, >0.  Zero only for the same index. */
static int cmp_key(float a, int64_t ia, float b, int64_t ib) {
  if (a < b) return -1;
  if (a > b) return 1;
  /* a == b as floats: only +0/-0 can still differ */
  int sa = signbit(a) ? 1 : 0, sb = signbit(b) ? 1 : 0;
  if (sa != sb) return sa ? -1 : 1;
  if (ia < ib) return -1;
  if (ia > ib) return 1;
  return 0;
}

/* Strict total order of records a and b in dimension d: by coordinate (as
 * float32 with -0 < +0, or as int32 / uint32), then by original index. */
static int cmp_rec(const pointset* P, int64_t a, int64_t b, int d) {
  if (P->ints) {
    int64_t x = icoord(P, a, d), y = icoord(P, b, d);
    if (x != y) return x < y ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
  }
  return cmp_key(coord(P, a, d), a, coord(P, b, d), b);
}

/* ---------------- plain merge sort of an index list by one dimension ----- */
static void merge_sort_idx(const pointset* P, int d, int64_t* a, int64_t* tmp, int64_t n) {
  if (n < 2) return;
  int64_t h = n / 2;
  merge_sort_idx(P, d, a, tmp, h);
  merge_sort_idx(P, d, a + h, tmp, n - h);
  int64_t i = 0, j = h, o = 0;
  while (i < h && j < n) {
    if (cmp_rec(P, a[j], a[i], d) < 0)
      tmp[o++] = a[j++];
    else
      tmp[o++] = a[i++];
  }
  while (i < h) tmp[o++] = a[i++];
  while (j < n) tmp[o++] = a[j++];
  memcpy(a, tmp, (size_t)n * sizeof *a);
}

/* Number of nodes of the subtree rooted at s in a level-order tree of N
 * nodes, counted level by level: the nodes j levels below s are the 2^j
 * consecutive slots starting at (s+1)*2^j - 1. */
int64_t kdo_subtree_size(int64_t s, int64_t N) {
  if (s < 0 || s >= N) return 0;
  int64_t total = 0, first = s, width = 1;
  while (first < N) {
    int64_t last = first + width; /* exclusive */
    if (last > N) last = N;
    total += last - first;
    first = 2 * first + 1;
    width *= 2;
  }
  return total;
}

static int widest_dim(const float* lo, const float* hi, int k) {
  int best = 0;
  float bestExt = hi[0] - lo[0];
  for (int d = 1; d < k; ++d) {
    float e = hi[d] - lo[d];
    if (e > bestExt) { bestExt = e; best = d; }
  }
  return best;
}

/* Scene bounding box under the strict order (-0 below +0). */
static void scene_box(const pointset* P, int64_t N, float* lo, float* hi) {
  for (int d = 0; d < P->k; ++d) {
    float l = coord(P, 0, d), h = l;
    for (int64_t i = 1; i < N; ++i) {
      float v = coord(P, i, d);
      if (cmp_key(v, 0, l, 0) < 0) l = v;
      if (cmp_key(v, 0, h, 0) > 0) h = v;
    }
    lo[d] = l;
    hi[d] = h;
  }
}

/* Tight bounding box of the records S[0..n), n >= 1 (float32 coordinates). */
static void tight_box(const pointset* P, const int64_t* S, int64_t n, float* lo, float* hi) {
  for (int d = 0; d < P->k; ++d) {
    float l = coord(P, S[0], d), h = l;
    for (int64_t i = 1; i < n; ++i) {
      float v = coord(P, S[i], d);
      if (cmp_key(v, 0, l, 0) < 0) l = v;
      if (cmp_key(v, 0, h, 0) > 0) h = v;
    }
    lo[d] = l;
    hi[d] = h;
  }
}

/* Widest side of the tight box of S[0..n): float32 extents as widest_dim,
 * or for integer coordinates the exact 64-bit extents max - min, scanned the
 * same way (strict '>' from d = 0). */
static int tight_widest(const pointset* P, const int64_t* S, int64_t n) {
  if (!P->ints) {
    float lo[KDO_MAXK], hi[KDO_MAXK];
    tight_box(P, S, n, lo, hi);
    return widest_dim(lo, hi, P->k);
  }
  int best = 0;
  int64_t bestExt = 0;
  for (int d = 0; d < P->k; ++d) {
    int64_t l = icoord(P, S[0], d), h = l;
    for (int64_t i = 1; i < n; ++i) {
      int64_t v = icoord(P, S[i], d);
      if (v < l) l = v;
      if (v > h) h = v;
    }
    int64_t e = h - l;
    if (d == 0 || e > bestExt) { bestExt = e; best = d; }
  }
  return best;
}

typedef struct {
  const pointset* P;
  int64_t N;
  int mode;
  int64_t* tmp;
  int32_t* orig_of_node; /* output: original index stored at node s */
} build_ctx;

static void build_rec(build_ctx* C, int64_t* S, int64_t n, int64_t s, int depth,
                      const float* lo, const float* hi) {
  if (n == 0) return;
  const int k = C->P->k;
  int d;
  if (C->mode == KDO_ROUND_ROBIN) {
    d = depth % k;
  } else if (C->mode == KDO_WIDEST) {
    d = widest_dim(lo, hi, k);
  } else { /* widest side of the box of this subtree's own points */
    d = tight_widest(C->P, S, n);
  }
  merge_sort_idx(C->P, d, S, C->tmp, n);
  int64_t p = kdo_subtree_size(2 * s + 1, C->N); /* Observation 1 */
  C->orig_of_node[s] = (int32_t)S[p];
  float x = C->P->ints ? 0.0f : coord(C->P, S[p], d); /* plane (clipped-domain rule only) */
  float clo[KDO_MAXK], chi[KDO_MAXK];
  memcpy(clo, lo, sizeof(float) * k);
  memcpy(chi, hi, sizeof(float) * k);
  chi[d] = x; /* left subtree's domain ends at the plane */
  build_rec(C, S, p, 2 * s + 1, depth + 1, clo, chi);
  chi[d] = hi[d];
  clo[d] = x; /* right subtree's domain starts at the plane */
  build_rec(C, S + p + 1, n - p - 1, 2 * s + 2, depth + 1, clo, chi);
}

static int check_args(const void* points, int64_t N, int k, int stride, int mode) {
  if (N < 0 || N > 2147483647LL) return KDO_INVALID;
  if (k < 1 || k > KDO_MAXK) return KDO_INVALID;
  if (stride < 4 * k || (stride % 4) != 0) return KDO_INVALID;
  if (mode & ~(0xFF | KDO_INT32 | KDO_UINT32)) return KDO_INVALID;
  if ((mode & KDO_INT32) && (mode & KDO_UINT32)) return KDO_INVALID;
  int split = mode & 0xFF;
  if (split != KDO_ROUND_ROBIN && split != KDO_WIDEST && split != KDO_WIDEST_TIGHT) return KDO_INVALID;
  if ((mode & (KDO_INT32 | KDO_UINT32)) && split == KDO_WIDEST) return KDO_INVALID;
  if (N > 0 && points == NULL) return KDO_INVALID;
  return KDO_OK;
}

static int has_nan(const pointset* P, int64_t N) {
  if (P->ints) return 0;
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < P->k; ++d)
      if (isnan(coord(P, i, d))) return 1;
  return 0;
}

/* Build the tree.  out_points (N * stride bytes, may be NULL) receives the
 * records in level order; out_orig (N int32, may be NULL) the original index
 * of the record at each node. */
int kdo_build(const void* points, int64_t N, int k, int stride, int mode,
              void* out_points, int32_t* out_orig) {
  int rc = check_args(points, N, k, stride, mode);
  if (rc) return rc;
  if (N == 0) return KDO_OK;
  pointset P = {(const unsigned char*)points, stride, k, coord_type(mode)};
  mode &= 0xFF;
  if (has_nan(&P, N)) return KDO_NAN;
  int64_t* S = (int64_t*)malloc((size_t)N * sizeof *S);
  int64_t* tmp = (int64_t*)malloc((size_t)N * sizeof *tmp);
  int32_t* orig = (int32_t*)malloc((size_t)N * sizeof *orig);
  if (!S || !tmp || !orig) { free(S); free(tmp); free(orig); return KDO_NOMEM; }
  for (int64_t i = 0; i < N; ++i) S[i] = i;
  float lo[KDO_MAXK] = {0}, hi[KDO_MAXK] = {0};
  if (!P.ints) scene_box(&P, N, lo, hi);
  build_ctx C = {&P, N, mode, tmp, orig};
  build_rec(&C, S, N, 0, 0, lo, hi);
  if (out_points) {
    unsigned char* o = (unsigned char*)out_points;
    for (int64_t s = 0; s < N; ++s)
      memcpy(o + s * stride, P.base + (int64_t)orig[s] * stride, (size_t)stride);
  }
  if (out_orig) memcpy(out_orig, orig, (size_t)N * sizeof *orig);
  free(S); free(tmp); free(orig);
  return KDO_OK;
}

/* ------------------------------------------------------------------------
 * The subtree below one node of a larger tree, built on its own: the same
 * recursion started at the node's depth (round robin continues with
 * dimension (first_dim + depth) mod k) and, for the clipped-domain rule, from
 * the node's domain (root_domain: k lower bounds, then k upper bounds).  A
 * subtree of a left-balanced complete tree is itself one of its size, so the
 * subtree's nodes in their own level order follow from Observation 1 exactly
 * as for a whole tree; ties still go by position in `points`.
 * ---------------------------------------------------------------------- */
int kdo_build_sub(const void* points, int64_t N, int k, int stride, int mode, int first_dim,
                  const float* root_domain, void* out_points, int32_t* out_orig) {
  int rc = check_args(points, N, k, stride, mode);
  if (rc) return rc;
  if (first_dim < 0 || first_dim >= k) return KDO_INVALID;
  if ((mode & 0xFF) == KDO_WIDEST && !root_domain) return KDO_INVALID;
  if (N == 0) return KDO_OK;
  pointset P = {(const unsigned char*)points, stride, k, coord_type(mode)};
  mode &= 0xFF;
  if (has_nan(&P, N)) return KDO_NAN;
  int64_t* S = (int64_t*)malloc((size_t)N * sizeof *S);
  int64_t* tmp = (int64_t*)malloc((size_t)N * sizeof *tmp);
  int32_t* orig = (int32_t*)malloc((size_t)N * sizeof *orig);
  if (!S || !tmp || !orig) { free(S); free(tmp); free(orig); return KDO_NOMEM; }
  for (int64_t i = 0; i < N; ++i) S[i] = i;
  float lo[KDO_MAXK] = {0}, hi[KDO_MAXK] = {0};
  if (mode == KDO_WIDEST)
    for (int d = 0; d < k; ++d) {
      lo[d] = root_domain[d];
      hi[d] = root_domain[k + d];
    }
  build_ctx C = {&P, N, mode, tmp, orig};
  build_rec(&C, S, N, 0, mode == KDO_ROUND_ROBIN ? first_dim : 0, lo, hi);
  if (out_points) {
    unsigned char* o = (unsigned char*)out_points;
    for (int64_t s = 0; s < N; ++s)
      memcpy(o + s * stride, P.base + (int64_t)orig[s] * stride, (size_t)stride);
  }
  if (out_orig) memcpy(out_orig, orig, (size_t)N * sizeof *orig);
  free(S); free(tmp); free(orig);
  return KDO_OK;
}

/* ------------------------------------------------------------------------
 * Invariant checker.  Given the input records, the built records and the
 * original index of each node, checks
 *   (1) orig is a permutation of [0,N) and out[s] is byte-identical to
 *       in[orig[s]];
 *   (2) the strict k-d condition: for every node i and every ancestor p,
 *       (x_d(i), orig(i)) < (x_d(p), orig(p)) if i lies in p's left subtree
 *       and > if in the right one, with d = p's split dimension.  For the
 *       widest mode the dimensions are recomputed top-down from the built
 *       tree's own planes and the scene box; for the tight-box mode from
 *       the box of each node's subtree in the built tree.
 * Because the left-balanced shape is implicit in the array layout and the
 * valid arrangement is unique under the strict order, (1) and (2) together
 * are equivalent to equality with kdo_build.  *first_bad receives the first
 * failing node (or -1).
 * ---------------------------------------------------------------------- */
int kdo_check(const void* in_points, const void* out_points, const int32_t* orig,
              int64_t N, int k, int stride, int mode, int64_t* first_bad) {
  int rc = check_args(in_points, N, k, stride, mode);
  if (first_bad) *first_bad = -1;
  if (rc) return rc;
  if (N == 0) return KDO_OK;
  pointset In = {(const unsigned char*)in_points, stride, k, coord_type(mode)};
  pointset Out = {(const unsigned char*)out_points, stride, k, coord_type(mode)};
  mode &= 0xFF;
  unsigned char* seen = (unsigned char*)calloc((size_t)N, 1);
  unsigned char* dim = (unsigned char*)malloc((size_t)N);
  if (!seen || !dim) { free(seen); free(dim); return KDO_NOMEM; }
  int64_t bad = -1;
  for (int64_t s = 0; s < N && bad < 0; ++s) {
    int64_t o = orig[s];
    if (o < 0 || o >= N || seen[o]) { bad = s; break; }
    seen[o] = 1;
    if (memcmp(In.base + o * stride, Out.base + s * stride, (size_t)stride) != 0) bad = s;
  }
  if (bad < 0) {
    if (mode == KDO_ROUND_ROBIN) {
      for (int64_t s = 0; s < N; ++s) {
        int lvl = 0;
        for (int64_t t = s + 1; t > 1; t >>= 1) ++lvl;
        dim[s] = (unsigned char)(lvl % k);
      }
    } else if (mode == KDO_WIDEST_TIGHT) {
      /* the records of node s's subtree, gathered by walking its levels */
      int64_t* sub = (int64_t*)malloc((size_t)N * sizeof *sub);
      if (!sub) { free(seen); free(dim); return KDO_NOMEM; }
      for (int64_t s = 0; s < N; ++s) {
        int64_t cnt = 0;
        for (int64_t first = s, width = 1; first < N; first = 2 * first + 1, width *= 2)
          for (int64_t t = first; t < first + width && t < N; ++t) sub[cnt++] = t;
        dim[s] = (unsigned char)tight_widest(&Out, sub, cnt);
      }
      free(sub);
    } else {
      /* top-down: the domain of node s is the scene box clipped by the
         planes of its ancestors; walk the path from the root each time */
      float lo0[KDO_MAXK], hi0[KDO_MAXK];
      scene_box(&Out, N, lo0, hi0);
      for (int64_t s = 0; s < N; ++s) {
        float lo[KDO_MAXK], hi[KDO_MAXK];
        memcpy(lo, lo0, sizeof(float) * k);
        memcpy(hi, hi0, sizeof(float) * k);
        int64_t path[64];
        int depth = 0;
        for (int64_t t = s; t > 0; t = (t - 1) / 2) path[depth++] = t;
        int64_t cur = 0;
        for (int j = depth - 1; j >= 0; --j) {
          int64_t child = path[j];
          int dc = dim[cur];
          float x = coord(&Out, cur, dc);
          if (child == 2 * cur + 1) hi[dc] = x; else lo[dc] = x;
          cur = child;
        }
        dim[s] = (unsigned char)widest_dim(lo, hi, k);
      }
    }
    for (int64_t i = 1; i < N && bad < 0; ++i) {
      int64_t child = i;
      for (int64_t p = (i - 1) / 2;; p = (p - 1) / 2) {
        int d = dim[p];
        /* the strict order on (coordinate, original index) of the two nodes */
        int c;
        if (Out.ints) {
          int64_t xi = icoord(&Out, i, d), xp = icoord(&Out, p, d);
          c = xi != xp ? (xi < xp ? -1 : 1) : (orig[i] < orig[p] ? -1 : (orig[i] > orig[p] ? 1 : 0));
        } else {
          c = cmp_key(coord(&Out, i, d), orig[i], coord(&Out, p, d), orig[p]);
        }
        int left = (child == 2 * p + 1);
        if ((left && c >= 0) || (!left && c <= 0)) { bad = i; break; }
        child = p;
        if (p == 0) break;
      }
    }
  }
  free(seen);
  free(dim);
  if (first_bad) *first_bad = bad;
  return bad < 0 ? KDO_OK : KDO_NOT_KD;
}

/* ------------------------------------------------------------------------
 * Single node, for sampled checks at sizes where the full recursive build is
 * too slow: follow the path root -> node, and at each step select the point of
 * rank ss(lChild) in the current subset (a plain quickselect under the strict
 * order), then keep the side the path continues into.  Same definition as
 * kdo_build (Observation 1 applied along one path).
 * ---------------------------------------------------------------------- */
static uint64_t lcg_next(uint64_t* st) {
  *st = *st * 6364136223846793005ULL + 1442695040888963407ULL;
  return *st >> 33;
}

/* Rearranges a[0..n) so that a[r] holds the rank-r element, lower ranks
 * before it and higher ranks after it. */
static void quickselect(const pointset* P, int d, int64_t* a, int64_t n, int64_t r) {
  uint64_t st = 0x9E3779B97F4A7C15ULL ^ (uint64_t)n;
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t pi = lo + (int64_t)(lcg_next(&st) % (uint64_t)(hi - lo + 1));
    int64_t piv = a[pi];
    a[pi] = a[hi];
    a[hi] = piv;
    int64_t store = lo;
    for (int64_t i = lo; i < hi; ++i) {
      if (cmp_rec(P, a[i], piv, d) < 0) {
        int64_t t = a[i]; a[i] = a[store]; a[store] = t;
        ++store;
      }
    }
    a[hi] = a[store];
    a[store] = piv;
    if (store == r) return;
    if (store < r) lo = store + 1; else hi = store - 1;
  }
}

int kdo_node(const void* points, int64_t N, int k, int stride, int mode, int64_t node,
             int32_t* out_orig) {
  int rc = check_args(points, N, k, stride, mode);
  if (rc) return rc;
  if (node < 0 || node >= N || !out_orig) return KDO_INVALID;
  pointset P = {(const unsigned char*)points, stride, k, coord_type(mode)};
  mode &= 0xFF;
  if (has_nan(&P, N)) return KDO_NAN;
  int64_t* S = (int64_t*)malloc((size_t)N * sizeof *S);
  if (!S) return KDO_NOMEM;
  for (int64_t i = 0; i < N; ++i) S[i] = i;
  float lo[KDO_MAXK] = {0}, hi[KDO_MAXK] = {0};
  if (!P.ints) scene_box(&P, N, lo, hi);
  int64_t path[64];
  int depth = 0;
  for (int64_t t = node; t > 0; t = (t - 1) / 2) path[depth++] = t;
  path[depth] = 0;
  int64_t s = 0, off = 0, n = N;
  int lvl = 0;
  for (int j = depth; j >= 0; --j) {
    s = path[j];
    int d;
    if (mode == KDO_ROUND_ROBIN) {
      d = lvl % k;
    } else if (mode == KDO_WIDEST) {
      d = widest_dim(lo, hi, k);
    } else {
      d = tight_widest(&P, S + off, n);
    }
    int64_t p = kdo_subtree_size(2 * s + 1, N);
    quickselect(&P, d, S + off, n, p);
    if (j == 0) {
      *out_orig = (int32_t)S[off + p];
      break;
    }
    float x = P.ints ? 0.0f : coord(&P, S[off + p], d);
    if (path[j - 1] == 2 * s + 1) {
      hi[d] = x;
      n = p;
    } else {
      lo[d] = x;
      off += p + 1;
      n = n - p - 1;
    }
    ++lvl;
  }
  free(S);
  return KDO_OK;
}
