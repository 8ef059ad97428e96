/* Host check of the CPU oracle (oracle/kd_oracle.c) and of the parallel CPU
 * port (oracle/paper_cpu.c) under AddressSanitizer and UndefinedBehavior-
 * Sanitizer: builds, invariant checks, the single-node selector and the
 * threaded port over edge sizes, every split rule, float32 / int32 / uint32
 * coordinates, payload strides, tie-heavy and extreme values, NaN input and
 * bad arguments.  Prints "OK <cases>" or the first failure.  Test
 * infrastructure; compiled and run by tests/test_oracle_sanitized.py. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int kdo_build(const void* points, int64_t N, int k, int stride, int mode, void* out_points,
              int32_t* out_orig);
int kdo_check(const void* in_points, const void* out_points, const int32_t* orig, int64_t N, int k,
              int stride, int mode, int64_t* first_bad);
int kdo_node(const void* points, int64_t N, int k, int stride, int mode, int64_t node,
             int32_t* out_orig);
int64_t kdo_subtree_size(int64_t s, int64_t N);
int pc_build(const void* points, int64_t N, int k, int stride, int mode, int threads, int32_t* out_orig);

enum { RR = 0, WIDEST = 1, TIGHT = 2, F_INT32 = 0x100, F_UINT32 = 0x200 };
enum { OK = 0, INVALID = 1, NAN_INPUT = 4 };

/* SplitMix64 (Steele, Lea and Flood 2014) */
static uint64_t g_state = 12345;
static uint64_t next64(void) {
  uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint32_t f2u(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* one coordinate's bits: pattern 0 spread values, 1 ties from a few values,
 * 2 the type's extremes */
static uint32_t coord_bits(int ctype, int pattern) {
  const uint64_t r = next64();
  if (ctype == 0) {
    static const float ties[] = {0.0f, 1.0f, 2.0f, -0.0f};
    const float ext[] = {-INFINITY, -3.4028235e38f, -1.0f, -0.0f, 0.0f, 1e-45f, 1.0f, 3.4028235e38f,
                         INFINITY};
    if (pattern == 0) return f2u((float)(r >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f);
    if (pattern == 1) return f2u(ties[r % 4]);
    return f2u(ext[r % 9]);
  }
  if (pattern == 0) return (uint32_t)(r >> 32);
  if (pattern == 1) return (uint32_t)(r % 3);
  {
    static const uint32_t ext[] = {0u, 1u, 0x7FFFFFFEu, 0x7FFFFFFFu, 0x80000000u, 0x80000001u,
                                   0xFFFFFFFEu, 0xFFFFFFFFu, 0x01000000u};
    return ext[r % 9];
  }
}

static int fail(const char* what, int64_t n, int k, int words, int mode, int pattern, long long got) {
  printf("FAIL %s: N=%lld k=%d words=%d mode=0x%x pattern=%d got=%lld\n", what, (long long)n, k,
         words, mode, pattern, got);
  return 1;
}

static int one_case(int64_t n, int k, int words, int ctype, int split, int pattern, long long* cases) {
  const int mode = split | (ctype == 1 ? F_INT32 : ctype == 2 ? F_UINT32 : 0);
  const int stride = 4 * words;
  uint32_t* in = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * stride);
  uint32_t* out = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * stride);
  int32_t* orig = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof *orig);
  int32_t* orig2 = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof *orig2);
  int bad = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int w = 0; w < words; ++w)
      in[i * words + w] = w < k ? coord_bits(ctype, pattern) : (uint32_t)next64();
  const int expect_invalid = split == WIDEST && ctype != 0;
  int rc = kdo_build(in, n, k, stride, mode, out, orig);
  ++*cases;
  if (expect_invalid) {
    bad = rc != INVALID ? fail("integer clipped domain accepted", n, k, words, mode, pattern, rc) : 0;
    goto done;
  }
  if (rc != OK) {
    bad = fail("kdo_build", n, k, words, mode, pattern, rc);
    goto done;
  }
  {
    int64_t first = -2;
    rc = kdo_check(in, out, orig, n, k, stride, mode, &first);
    if (rc != OK || first != -1) {
      bad = fail("kdo_check of the oracle's own tree", n, k, words, mode, pattern, first);
      goto done;
    }
  }
  for (int t = 0; t < 4 && n > 0; ++t) {
    const int64_t s = (int64_t)(next64() % (uint64_t)n);
    int32_t o = -1;
    rc = kdo_node(in, n, k, stride, mode, s, &o);
    if (rc != OK || o != orig[s]) {
      bad = fail("kdo_node", n, k, words, mode, pattern, o);
      goto done;
    }
  }
  for (int threads = 1; threads <= 3; threads += 2) {
    memset(orig2, 0xFF, (size_t)(n > 0 ? n : 1) * sizeof *orig2);
    rc = pc_build(in, n, k, stride, mode, threads, orig2);
    if (rc != OK || (n > 0 && memcmp(orig, orig2, (size_t)n * sizeof *orig) != 0)) {
      bad = fail("pc_build against the oracle", n, k, words, mode, pattern, rc);
      goto done;
    }
  }
  if (n >= 3) {  /* planted: the root's two children swapped */
    int64_t first = -2;
    uint32_t tmp[64];
    memcpy(tmp, out + words, stride);
    memcpy(out + words, out + 2 * words, stride);
    memcpy(out + 2 * words, tmp, stride);
    const int32_t t = orig[1];
    orig[1] = orig[2];
    orig[2] = t;
    rc = kdo_check(in, out, orig, n, k, stride, mode, &first);
    if (first < 0) bad = fail("planted swap not found", n, k, words, mode, pattern, first);
  }
done:
  free(in);
  free(out);
  free(orig);
  free(orig2);
  return bad;
}

int main(void) {
  long long cases = 0;
  static const int64_t sizes[] = {0, 1, 2, 3, 5, 8, 31, 100, 1000, 4097};
  static const int ks[] = {1, 2, 3, 4, 8};
  for (size_t a = 0; a < sizeof sizes / sizeof *sizes; ++a)
    for (size_t b = 0; b < sizeof ks / sizeof *ks; ++b)
      for (int extra = 0; extra <= 2; extra += 2)
        for (int ctype = 0; ctype < 3; ++ctype)
          for (int split = 0; split < 3; ++split)
            for (int pattern = 0; pattern < 3; ++pattern) {
              const int64_t n = ks[b] == 8 && sizes[a] > 1000 ? 1000 : sizes[a];
              if (one_case(n, ks[b], ks[b] + extra, ctype, split, pattern, &cases)) return 1;
            }

  /* NaN input: refused by both builders */
  {
    float pts[30];
    for (int i = 0; i < 30; ++i) pts[i] = (float)i;
    pts[17] = NAN;
    float out[30];
    int32_t orig[10];
    int rc = kdo_build(pts, 10, 3, 12, RR, out, orig);
    if (rc != NAN_INPUT) return fail("NaN accepted by the oracle", 10, 3, 3, RR, 0, rc);
    rc = pc_build(pts, 10, 3, 12, RR, 2, orig);
    if (rc == OK) return fail("NaN accepted by the CPU port", 10, 3, 3, RR, 0, rc);
    /* the same bits as int32 / uint32 are ordinary integers */
    if (kdo_build(pts, 10, 3, 12, RR | F_INT32, out, orig) != OK ||
        kdo_build(pts, 10, 3, 12, RR | F_UINT32, out, orig) != OK)
      return fail("NaN bits refused as integers", 10, 3, 3, RR, 0, -1);
    cases += 4;
  }
  /* bad arguments */
  {
    float pts[24] = {0};
    float out[24];
    int32_t orig[8];
    const struct { int64_t n; int k, stride, mode; } bad[] = {
        {-1, 3, 12, RR}, {8, 0, 12, RR}, {8, 9, 36, RR}, {8, 3, 8, RR}, {8, 3, 14, RR},
        {8, 3, 12, 5}, {8, 3, 12, RR | F_INT32 | F_UINT32}, {8, 3, 12, WIDEST | F_UINT32},
        {8, 3, 12, RR | 0x400}};
    for (size_t i = 0; i < sizeof bad / sizeof *bad; ++i) {
      if (kdo_build(pts, bad[i].n, bad[i].k, bad[i].stride, bad[i].mode, out, orig) != INVALID)
        return fail("bad argument accepted", bad[i].n, bad[i].k, bad[i].stride / 4, bad[i].mode, 0, i);
      ++cases;
    }
    if (kdo_build(NULL, 8, 3, 12, RR, out, orig) != INVALID)
      return fail("NULL points accepted", 8, 3, 3, RR, 0, -1);
  }
  /* subtree sizes: the whole tree, and 1 + both children everywhere */
  for (int64_t n = 1; n <= 300; ++n) {
    if (kdo_subtree_size(0, n) != n) return fail("ss(0)", n, 0, 0, 0, 0, kdo_subtree_size(0, n));
    for (int64_t s = 0; s < n; ++s)
      if (kdo_subtree_size(s, n) != 1 + kdo_subtree_size(2 * s + 1, n) + kdo_subtree_size(2 * s + 2, n))
        return fail("ss recursion", n, 0, 0, 0, 0, s);
    cases += n;
  }
  printf("OK %lld\n", cases);
  return 0;
}
