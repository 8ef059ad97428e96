// Host-side check of the level layout used by the CUDA kernels
// (paper_2211_00120_gb300/csrc/kdb_internal.cuh) against subtree sizes
// counted level by level, for every N in [1, NMAX].  Prints "OK <cases>" or
// the first mismatch.  Test infrastructure; compiled by tests/test_index_math.py.
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kdb_internal.cuh"

static long long counted_size(long long s, long long n) {
  if (s >= n) return 0;
  long long total = 0, first = s, width = 1;
  while (first < n) {
    long long last = first + width < n ? first + width : n;
    total += last - first;
    first = 2 * first + 1;
    width *= 2;
  }
  return total;
}

int main(int argc, char** argv) {
  const long long NMAX = argc > 1 ? atoll(argv[1]) : 3000;
  long long cases = 0;
  for (long long n = 1; n <= NMAX; ++n) {
    const kdb::Tree t = kdb::make_tree((uint32_t)n);
    int L = 0;
    while ((1LL << L) - 1 < n) ++L;  // smallest L with 2^L - 1 >= n
    if (t.L != L) { printf("FAIL L n=%lld got %d want %d\n", n, t.L, L); return 1; }
    for (long long s = 0; s < n + 2; ++s) {
      if ((long long)kdb::subtree_size(t, (uint32_t)s) != counted_size(s, n)) {
        printf("FAIL ss n=%lld s=%lld\n", n, s);
        return 1;
      }
    }
    for (int l = 0; l + 2 <= L; ++l) {
      const kdb::LevelLayout y = kdb::LevelLayout::make(t, l);
      const long long F = (1LL << l) - 1;
      if ((long long)y.items != n - F) { printf("FAIL items n=%lld l=%d\n", n, l); return 1; }
      long long pos = 0, lefts = 0;
      for (long long sr = 0; sr < (1LL << l); ++sr) {
        if (y.h >= 1 && (long long)y.left_before((uint32_t)sr) != lefts) {
          printf("FAIL left_before n=%lld l=%d s_rel=%lld\n", n, l, sr);
          return 1;
        }
        lefts += counted_size(2 * (F + sr) + 1, n);
        const long long s = F + sr;
        const long long size = counted_size(s, n);
        if ((long long)y.seg_start((uint32_t)sr) != pos) {
          printf("FAIL start n=%lld l=%d s=%lld\n", n, l, s);
          return 1;
        }
        if ((long long)y.left_size((uint32_t)sr) != counted_size(2 * s + 1, n)) {
          printf("FAIL left n=%lld l=%d s=%lld\n", n, l, s);
          return 1;
        }
        for (long long j = pos; j < pos + size; ++j)
          if ((long long)y.seg_of((uint32_t)j) != sr) {
            printf("FAIL seg_of n=%lld l=%d j=%lld\n", n, l, j);
            return 1;
          }
        pos += size;
        ++cases;
      }
      if (pos != n - F) { printf("FAIL total n=%lld l=%d\n", n, l); return 1; }
      if (y.h >= 1 && (long long)y.left_before((uint32_t)(1LL << l)) != lefts) {
        printf("FAIL left_before end n=%lld l=%d\n", n, l);
        return 1;
      }
    }
  }
  // float_key is monotone and -0 < +0
  const float vals[] = {-INFINITY, -3.5f, -1e-40f, -0.0f, 0.0f, 1e-40f, 1.0f, 2.5e30f, INFINITY};
  for (unsigned i = 0; i + 1 < sizeof vals / sizeof vals[0]; ++i) {
    uint32_t a, b;
    memcpy(&a, &vals[i], 4);
    memcpy(&b, &vals[i + 1], 4);
    if (!(kdb::float_key(a) < kdb::float_key(b)) || kdb::key_to_float_bits(kdb::float_key(a)) != a) {
      printf("FAIL float_key %u\n", i);
      return 1;
    }
  }
  // the coordinate key maps of the three coordinate types: each inverts
  // exactly (every third bit pattern, a stride coprime to 2^32) and orders
  // keys as the type orders values (random pairs): float32 by value with
  // -0 < +0 (NaN excluded), int32 signed, uint32 unsigned
  for (int ctype = 0; ctype < 3; ++ctype) {
    for (uint64_t u = 0; u < (1ull << 32); u += 3) {
      const uint32_t b = (uint32_t)u;
      if (ctype == kdb::kCoordF32 && (b & 0x7FFFFFFFu) > 0x7F800000u) continue;
      if (kdb::key_to_coord_bits(kdb::coord_key(b, ctype), ctype) != b) {
        printf("FAIL key inverse type %d bits %u\n", ctype, b);
        return 1;
      }
    }
    uint64_t st = 0x1234567ull + (uint64_t)ctype;
    auto rnd = [&st]() {  // SplitMix64 (Steele, Lea and Flood 2014)
      uint64_t z = (st += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    for (int t = 0; t < 20000000; ++t) {
      const uint64_t r = rnd();
      uint32_t a = (uint32_t)r, b = (uint32_t)(r >> 32);
      if (t % 4 == 0) b = a ^ (1u << (rnd() % 32));  // near pairs
      if (ctype == kdb::kCoordF32 && (((a & 0x7FFFFFFFu) > 0x7F800000u) || ((b & 0x7FFFFFFFu) > 0x7F800000u)))
        continue;
      bool less;
      if (ctype == kdb::kCoordF32) {
        float fa, fb;
        memcpy(&fa, &a, 4);
        memcpy(&fb, &b, 4);
        less = fa < fb || (fa == fb && std::signbit(fa) && !std::signbit(fb));
      } else if (ctype == kdb::kCoordI32) {
        less = (int32_t)a < (int32_t)b;
      } else {
        less = a < b;
      }
      if (less != (kdb::coord_key(a, ctype) < kdb::coord_key(b, ctype))) {
        printf("FAIL key order type %d %u %u\n", ctype, a, b);
        return 1;
      }
      ++cases;
    }
  }
  printf("OK %lld\n", cases);
  return 0;
}
