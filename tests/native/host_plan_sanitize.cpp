// Host check of the library's host-side code under AddressSanitizer and
// UndefinedBehaviorSanitizer: build plans (workspace layout of single and
// batched builds over many sizes, dimensions, strides and modes, valid and
// invalid), the tile-shape tables and setting, and the tuning-file parser on
// random input.  Calls nothing that needs a GPU.  Prints "OK <cases>" or the
// first failure.  Test infrastructure; compiled and run by
// tests/test_host_sanitized.py.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "kdb.h"

static uint64_t g_state = 99;
static uint64_t next64() {  // SplitMix64 (Steele, Lea and Flood 2014)
  uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static int fail(const char* what, long long a, long long b) {
  std::printf("FAIL %s: %lld %lld\n", what, a, b);
  return 1;
}

int main(int argc, char** argv) {
  const std::string tmp = argc > 1 ? argv[1] : "host_plan_sanitize.json";
  long long cases = 0;
  const int modes[] = {KDB_SPLIT_ROUND_ROBIN, KDB_SPLIT_WIDEST_EXTENT, KDB_SPLIT_WIDEST_TIGHT};
  const int types[] = {0, KDB_COORDS_INT32, KDB_COORDS_UINT32, KDB_COORDS_INT32 | KDB_COORDS_UINT32};
  const int64_t sizes[] = {-1, 0, 1, 2, 3, 7, 8, 100, 8191, 8192, 12289, 100000, 1 << 20, 5000011,
                           100000000, 2147483647LL, 2147483648LL};

  // single builds: every combination sizes a workspace or is refused
  for (int64_t n : sizes)
    for (int k = 0; k <= 9; ++k)
      for (int extra = 0; extra <= 2; ++extra)
        for (int m : modes)
          for (int t : types) {
            const int stride = 4 * k + 4 * extra;
            const size_t ws = kdb_workspace_size(n, k, stride, (kdb_split_mode)(m | t));
            const bool valid = n >= 0 && n <= 2147483647LL && k >= 1 && k <= 8 && stride >= 4 * k &&
                               t != (KDB_COORDS_INT32 | KDB_COORDS_UINT32) &&
                               !(t && m == KDB_SPLIT_WIDEST_EXTENT) &&
                               !(m == KDB_SPLIT_WIDEST_TIGHT && k > 3);
            if (!valid && ws != 0) return fail("invalid build sized", n, k);
            if (valid && n > 1 && ws == 0) return fail("valid build not sized", n, k);
            ++cases;
          }

  // batched builds: random set tables, some of them malformed
  for (int trial = 0; trial < 3000; ++trial) {
    const int sets = 1 + (int)(next64() % 200);
    std::vector<int64_t> offs(sets + 1, 0);
    for (int b = 0; b < sets; ++b) {
      const uint64_t r = next64();
      int64_t sz = (r & 3) == 0 ? (int64_t)(r % 3) : (int64_t)((r >> 8) % ((r & 4) ? 20000 : 300));
      offs[b + 1] = offs[b] + sz;
    }
    int bad = (int)(next64() % 8);
    if (bad == 1) offs[0] = 5;
    if (bad == 2 && sets > 1) offs[1] = offs[2] + 1;  // decreasing
    if (bad == 2 && sets == 1) bad = 0;                // nothing changed
    if (bad == 3) offs[sets] = -1;
    const int k = 1 + (int)(next64() % 8);
    const int m = modes[next64() % 3];
    const size_t ws = kdb_batched_workspace_size(offs.data(), sets, k, 4 * k, (kdb_split_mode)m);
    if (bad >= 1 && bad <= 3 && ws != 0) return fail("malformed set table sized", trial, bad);
    ++cases;
  }
  if (kdb_batched_workspace_size(nullptr, 3, 3, 12, KDB_SPLIT_ROUND_ROBIN) != 0)
    return fail("NULL set table sized", 0, 0);

  // tile shapes, digit widths and the process-wide setting
  for (int kernel = -1; kernel <= 3; ++kernel) {
    const int count = kdb_tuning_shape_count(kernel);
    const bool known = kernel == KDB_TUNE_PARTITION || kernel == KDB_TUNE_RADIX || kernel == KDB_TUNE_DIGITS;
    if (known != (count > 0)) return fail("shape count", kernel, count);
    for (int i = -1; i <= count + 1; ++i) {
      int th = 0, it = 0, bl = 0;
      const kdb_status s = kdb_tuning_shape(kernel, i, &th, &it, &bl);
      if ((s == KDB_OK) != (count > 0 && i >= 0 && i < count)) return fail("shape lookup", kernel, i);
      ++cases;
    }
  }
  for (int p = -1; p <= 4; ++p)
    for (int r = -1; r <= 3; ++r)
      for (int bits = 5; bits <= 9; ++bits) {
        const kdb_tuning t{p, r, bits};
        const kdb_status s = kdb_set_tuning(&t);
        kdb_tuning g{};
        kdb_get_tuning(&g);
        if (s == KDB_OK && (g.partition_shape != p || g.radix_shape != r || g.digit_bits != bits))
          return fail("set/get", p, r);
        if (s == KDB_OK) {
          if (kdb_save_tuning(tmp.c_str()) != KDB_OK) return fail("save", p, r);
          const kdb_tuning z{0, 0, 8};
          kdb_set_tuning(&z);
          if (kdb_load_tuning(tmp.c_str()) != KDB_OK) return fail("load", p, r);
          kdb_get_tuning(&g);
          if (g.partition_shape != p || g.radix_shape != r || g.digit_bits != bits) return fail("round trip", p, r);
        }
        ++cases;
      }
  {
    const kdb_tuning z{0, 0, 8};
    kdb_set_tuning(&z);
  }
  // the table: lookups by kind, and a file holding it
  kdb_clear_tuning_table();
  for (int64_t n : {(int64_t)0, (int64_t)1, (int64_t)1000, (int64_t)1 << 40}) {
    kdb_tuning g{};
    int hit = 7;
    if (kdb_lookup_tuning(n, 3, 12, KDB_SPLIT_ROUND_ROBIN, &g, &hit) != KDB_OK || hit != 0 || g.digit_bits != 8)
      return fail("lookup of an empty table", (int)n, hit);
    ++cases;
  }
  if (kdb_lookup_tuning(10, 3, 12, KDB_SPLIT_ROUND_ROBIN, nullptr, nullptr) != KDB_ERR_INVALID_ARGUMENT)
    return fail("lookup into NULL", 0, 0);
  {
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail("temp file", 0, 0);
    std::fputs("{\"partition\": [256, 13, 4], \"radix\": [256, 13, 3], \"digit_bits\": 8, \"table\": ["
               "{\"log2n\": 27, \"k\": 3, \"stride\": 12, \"mode\": 0, \"partition\": [256, 13, 4], "
               "\"radix\": [256, 13, 3], \"digit_bits\": 6}]}", f);
    std::fclose(f);
    if (kdb_load_tuning(tmp.c_str()) != KDB_OK) return fail("table load", 0, 0);
    kdb_tuning g{};
    int hit = 0;
    kdb_lookup_tuning(100000000, 3, 12, KDB_SPLIT_ROUND_ROBIN, &g, &hit);
    if (!hit || g.digit_bits != 6) return fail("table entry", hit, g.digit_bits);
    kdb_lookup_tuning(100000000, 3, 16, KDB_SPLIT_ROUND_ROBIN, &g, &hit);
    if (hit || g.digit_bits != 8) return fail("other stride", hit, g.digit_bits);
    kdb_clear_tuning_table();
    kdb_lookup_tuning(100000000, 3, 12, KDB_SPLIT_ROUND_ROBIN, &g, &hit);
    if (hit) return fail("cleared table", hit, 0);
    cases += 3;
  }

  // the tuning-file parser on random bytes and on mutated valid files
  const std::string good =
      "{\"partition\": [256, 13, 4], \"radix\": [256, 13, 3], \"digit_bits\": 6, \"table\": [{\"log2n\": 20, "
      "\"k\": 2, \"stride\": 8, \"mode\": 1, \"partition\": [512, 13, 2], \"radix\": [512, 8, 2], "
      "\"digit_bits\": 8}]}";
  for (int trial = 0; trial < 3000; ++trial) {
    std::string s;
    if (trial % 3 == 0) {
      const size_t len = next64() % 300;
      for (size_t i = 0; i < len; ++i) s.push_back((char)(next64() & 255));
    } else {
      s = good;
      const int edits = 1 + (int)(next64() % 5);
      for (int e = 0; e < edits && !s.empty(); ++e) {
        const size_t p = next64() % s.size();
        switch (next64() % 3) {
          case 0: s.erase(p, 1); break;
          case 1: s.insert(p, 1, "0123456789,[]{}\": -+"[next64() % 20]); break;
          default: s.resize(p); break;
        }
      }
    }
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail("temp file", trial, 0);
    std::fwrite(s.data(), 1, s.size(), f);
    std::fclose(f);
    const kdb_status st = kdb_load_tuning(tmp.c_str());
    if (st != KDB_OK && st != KDB_ERR_INVALID_ARGUMENT) return fail("load status", trial, st);
    kdb_tuning g{};
    kdb_get_tuning(&g);
    if (g.partition_shape < 0 || g.partition_shape >= kdb_tuning_shape_count(KDB_TUNE_PARTITION) ||
        g.radix_shape < 0 || g.radix_shape >= kdb_tuning_shape_count(KDB_TUNE_RADIX) ||
        (g.digit_bits != 8 && g.digit_bits != 6))
      return fail("setting out of range", g.partition_shape, g.radix_shape);
    int hit = 0;
    if (kdb_lookup_tuning(1 << 19, 2, 8, (kdb_split_mode)1, &g, &hit) != KDB_OK ||
        (hit && (g.partition_shape < 0 || g.partition_shape >= kdb_tuning_shape_count(KDB_TUNE_PARTITION) ||
                 g.radix_shape < 0 || g.radix_shape >= kdb_tuning_shape_count(KDB_TUNE_RADIX))))
      return fail("table entry out of range", trial, hit);
    ++cases;
  }
  std::remove(tmp.c_str());
  if (kdb_load_tuning(nullptr) != KDB_ERR_INVALID_ARGUMENT) return fail("NULL path", 0, 0);
  for (int code = -1; code <= 9; ++code)
    if (!kdb_status_string((kdb_status)code)) return fail("status string", code, 0);
  std::printf("OK %lld\n", cases);
  return 0;
}
