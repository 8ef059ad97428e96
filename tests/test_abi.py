"""The C-ABI library builds for sm_103a, loads, and exports exactly what
include/kdb.h declares.  Only calls that need no GPU are made here: argument
checking, workspace sizing and status strings."""
import ctypes
import json
import subprocess

import pytest

from paper_2211_00120_gb300 import build_lib, kdb


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return kdb.load()


def test_exports_every_declared_symbol(lib):
    declared = kdb.declared_symbols()
    assert {"kdb_build", "kdb_build_batched", "kdb_validate", "kdb_build_ex",
            "kdb_workspace_size", "kdb_status_string", "kdb_build_host"} <= set(declared)
    out = subprocess.run(["nm", "-D", "--defined-only", kdb.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split()[-1].startswith("kdb_")}
    assert exported == set(declared)
    for name in declared:
        assert getattr(lib, name) is not None


def test_status_strings(lib):
    for code in range(8):
        assert lib.kdb_status_string(code)
    assert lib.kdb_status_string(0) == b"ok"
    assert lib.kdb_version() >= 100


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    bad = [
        (-1, 3, 12),    # negative N
        (1 << 31, 3, 12),  # N above 2^31-1
        (10, 0, 12),    # k < 1
        (10, 9, 36),    # k > 8
        (10, 3, 8),     # stride < 4k
        (10, 3, 14),    # stride not a multiple of 4
    ]
    for n, k, stride in bad:
        assert lib.kdb_build(ctypes.c_void_p(16), n, k, stride, 0, None) == kdb.ERR_INVALID_ARGUMENT
        assert lib.kdb_workspace_size(n, k, stride, 0) == 0
    assert lib.kdb_build(ctypes.c_void_p(16), 10, 3, 12, 7, None) == kdb.ERR_INVALID_ARGUMENT
    assert lib.kdb_build(None, 10, 3, 12, 0, None) == kdb.ERR_INVALID_ARGUMENT
    assert lib.kdb_build(ctypes.c_void_p(18), 10, 3, 12, 0, None) == kdb.ERR_INVALID_ARGUMENT
    offs = (ctypes.c_int64 * 3)(0, 5, 3)  # decreasing offsets
    assert lib.kdb_build_batched(ctypes.c_void_p(16), offs, 2, 3, 12, 0, None) == \
        kdb.ERR_INVALID_ARGUMENT


def test_trivial_sizes_need_no_work(lib):
    # N <= 1 returns immediately (no device call is made for N = 0)
    assert lib.kdb_build(None, 0, 3, 12, 0, None) == kdb.OK
    assert lib.kdb_workspace_size(1, 3, 12, 0) == 0


def test_workspace_size_grows_with_n(lib):
    a = lib.kdb_workspace_size(1000, 3, 12, 0)
    b = lib.kdb_workspace_size(100000, 3, 12, 0)
    c = lib.kdb_workspace_size(100000, 3, 12, 1)
    # the split rules differ in their extras (round robin: a second set of
    # look-back words for its tagged pass; widest: the domains)
    assert 0 < a < b and a < c and abs(b - c) < 0.05 * b
    # linear in N: under 256 bytes per point at these sizes (three lists of
    # 16-byte entries, double-buffered, dominate)
    assert b < 256 * 100000
    assert lib.kdb_workspace_size(1000000, 3, 12, 0) < 10 * b


def test_placement_setting_round_trips(lib):
    prev = kdb.kdb_set_placement(kdb.PLACEMENT_IN_PLACE)
    try:
        assert prev == kdb.PLACEMENT_AUTO
        assert kdb.kdb_set_placement(7) == kdb.PLACEMENT_IN_PLACE  # invalid: unchanged
        assert kdb.kdb_set_placement(kdb.PLACEMENT_AUTO) == kdb.PLACEMENT_IN_PLACE
    finally:
        kdb.kdb_set_placement(kdb.PLACEMENT_AUTO)


def test_tuning_shapes_and_setting_round_trip(lib):
    part = kdb.kdb_tuning_shapes(kdb.TUNE_PARTITION)
    rad = kdb.kdb_tuning_shapes(kdb.TUNE_RADIX)
    assert len(part) >= 2 and len(rad) >= 2
    for threads, items, blocks in part + rad:
        assert threads % 32 == 0 and items > 0 and blocks > 0
        # a tile of either sort kernel spans at most two subtrees of a global
        # level (subtrees there hold at least 2^13 - 1 points)
        assert threads * items < (1 << 13) - 1
    assert part[0] == (256, 13, 4) and rad[0] == (256, 13, 3)  # the defaults
    # digit widths: (bits, passes per 32-bit key, 1), 8 bits first
    assert kdb.kdb_tuning_shapes(kdb.TUNE_DIGITS) == [(8, 4, 1), (6, 6, 1)]
    assert kdb.kdb_digit_widths() == [8, 6]
    assert lib.kdb_tuning_shape_count(9) == -1
    assert lib.kdb_tuning_shape(kdb.TUNE_RADIX, len(rad), None, None, None) == kdb.ERR_INVALID_ARGUMENT
    assert lib.kdb_tuning_shape(kdb.TUNE_DIGITS, 2, None, None, None) == kdb.ERR_INVALID_ARGUMENT
    assert kdb.kdb_get_tuning() == (0, 0, 8)
    try:
        kdb.kdb_set_tuning(len(part) - 1, len(rad) - 1, 6)
        assert kdb.kdb_get_tuning() == (len(part) - 1, len(rad) - 1, 6)
        for bad in [(len(part), 0, 8), (0, -1, 8), (0, 0, 7), (0, 0, 11)]:
            with pytest.raises(kdb.KdbError):
                kdb.kdb_set_tuning(*bad)  # out of range or not compiled: unchanged
        assert kdb.kdb_get_tuning() == (len(part) - 1, len(rad) - 1, 6)
    finally:
        kdb.kdb_set_tuning(0, 0)


def test_tuning_table_lookup_by_kind(lib, tmp_path):
    """A table entry applies to its kind only: the same bit length of N, k,
    stride and mode argument; everything else takes the process-wide
    setting."""
    part = kdb.kdb_tuning_shapes(kdb.TUNE_PARTITION)
    rad = kdb.kdb_tuning_shapes(kdb.TUNE_RADIX)
    f = tmp_path / "table.json"
    entry = {"log2n": 27, "k": 3, "stride": 12, "mode": 0, "partition": list(part[1]),
             "radix": list(rad[1]), "digit_bits": 6}
    try:
        kdb.kdb_clear_tuning_table()
        assert kdb.kdb_lookup_tuning(10**8, 3, 12) == ((0, 0, 8), False)
        f.write_text(json.dumps({"partition": list(part[0]), "radix": list(rad[0]), "table": [entry]}))
        kdb.kdb_load_tuning(str(f))
        assert kdb.kdb_lookup_tuning(10**8, 3, 12) == ((1, 1, 6), True)  # 1e8 has 27 bits
        assert kdb.kdb_lookup_tuning(2**26, 3, 12) == ((1, 1, 6), True)
        for other in [(2**27, 3, 12, 0), (2**26 - 1, 3, 12, 0), (10**8, 2, 12, 0), (10**8, 3, 16, 0),
                      (10**8, 3, 12, kdb.WIDEST_EXTENT), (10**8, 3, 12, kdb.COORDS_INT32)]:
            assert kdb.kdb_lookup_tuning(*other) == ((0, 0, 8), False), other
        kdb.kdb_set_tuning(2, 1, 6)  # the process-wide setting moves the rest only
        assert kdb.kdb_lookup_tuning(10**8, 3, 16) == ((2, 1, 6), False)
        assert kdb.kdb_lookup_tuning(10**8, 3, 12) == ((1, 1, 6), True)
        # saved with the setting, replaced whole on load
        kdb.kdb_save_tuning(str(f))
        j = json.loads(f.read_text())
        assert j["digit_bits"] == 6 and j["table"] == [entry]
        kdb.kdb_clear_tuning_table()
        kdb.kdb_set_tuning(0, 0)
        kdb.kdb_load_tuning(str(f))
        assert kdb.kdb_get_tuning() == (2, 1, 6)
        assert kdb.kdb_lookup_tuning(10**8, 3, 12) == ((1, 1, 6), True)
        # a repeated kind: the later entry wins
        later = dict(entry, digit_bits=8)
        f.write_text(json.dumps({"partition": list(part[0]), "radix": list(rad[0]), "table": [entry, later]}))
        kdb.kdb_load_tuning(str(f))
        assert kdb.kdb_lookup_tuning(10**8, 3, 12) == ((1, 1, 8), True)
        # a bad entry refuses the whole file
        for bad in [dict(entry, digit_bits=7), dict(entry, k=9), dict(entry, log2n=-1),
                    dict(entry, radix=[96, 7, 5]), {"k": 3}]:
            f.write_text(json.dumps({"partition": list(part[0]), "radix": list(rad[0]), "table": [bad]}))
            with pytest.raises(kdb.KdbError):
                kdb.kdb_load_tuning(str(f))
        f.write_text(json.dumps({"partition": list(part[0]), "radix": list(rad[0]), "table": [entry] * 257}))
        with pytest.raises(kdb.KdbError):
            kdb.kdb_load_tuning(str(f))
        assert kdb.kdb_lookup_tuning(10**8, 3, 12) == ((1, 1, 8), True)
        with pytest.raises(kdb.KdbError):
            kdb.kdb_lookup_tuning(-1, 3, 12)
    finally:
        kdb.kdb_clear_tuning_table()
        kdb.kdb_set_tuning(0, 0)


def test_tuning_file_round_trip_and_refusals(lib, tmp_path):
    part = kdb.kdb_tuning_shapes(kdb.TUNE_PARTITION)
    rad = kdb.kdb_tuning_shapes(kdb.TUNE_RADIX)
    f = tmp_path / "tuning.json"
    try:
        kdb.kdb_clear_tuning_table()
        kdb.kdb_set_tuning(2, 1)
        kdb.kdb_save_tuning(str(f))
        j = json.loads(f.read_text())
        assert j == {"partition": list(part[2]), "radix": list(rad[1]), "digit_bits": 8, "table": []}
        kdb.kdb_set_tuning(0, 0, 6)
        kdb.kdb_load_tuning(str(f))
        assert kdb.kdb_get_tuning() == (2, 1, 8)
        # shapes are matched by value: a shape this library does not carry,
        # a malformed file or a missing one is refused and changes nothing
        bad = [{"partition": [96, 7, 5], "radix": list(rad[0])},
               {"partition": list(part[0])},
               {"partition": list(part[0]), "radix": [256, 13]},
               {"partition": list(part[0]), "radix": list(rad[0]), "digit_bits": 11},
               {"partition": list(part[0]), "radix": list(rad[0]), "table": {}}]
        for b in bad:
            f.write_text(json.dumps(b))
            with pytest.raises(kdb.KdbError):
                kdb.kdb_load_tuning(str(f))
        for text in ["not json", json.dumps({"partition": list(part[0]), "radix": list(rad[0])}) + " x"]:
            f.write_text(text)
            with pytest.raises(kdb.KdbError):
                kdb.kdb_load_tuning(str(f))
        with pytest.raises(kdb.KdbError):
            kdb.kdb_load_tuning(str(tmp_path / "missing.json"))
        assert kdb.kdb_get_tuning() == (2, 1, 8)
        # whitespace and key order are free; the width defaults to 8 bits
        f.write_text('{ "radix" : [ %d , %d , %d ] ,\n "partition":[%d,%d,%d] }' % (rad[0] + part[1]))
        kdb.kdb_set_tuning(0, 0, 6)
        kdb.kdb_load_tuning(str(f))
        assert kdb.kdb_get_tuning() == (1, 0, 8)
    finally:
        kdb.kdb_set_tuning(0, 0)


def test_uint32_flag_and_its_refusals(lib):
    assert kdb.COORDS_UINT32 == 0x200
    # a valid combination sizes a workspace; both flags, or uint32 with the
    # clipped-domain rule, are invalid (size 0)
    assert lib.kdb_workspace_size(100000, 3, 12, kdb.ROUND_ROBIN | kdb.COORDS_UINT32) > 0
    assert lib.kdb_workspace_size(100000, 3, 12, kdb.WIDEST_TIGHT | kdb.COORDS_UINT32) > 0
    assert lib.kdb_workspace_size(100000, 3, 12, kdb.WIDEST_EXTENT | kdb.COORDS_UINT32) == 0
    assert lib.kdb_workspace_size(100000, 3, 12, kdb.COORDS_UINT32 | kdb.COORDS_INT32) == 0


def test_binding_sets_the_coordinate_type_from_the_dtype():
    import torch

    f = torch.zeros(4, 3, dtype=torch.float32)
    i = torch.zeros(4, 3, dtype=torch.int32)
    assert kdb._mode(f, kdb.ROUND_ROBIN) == kdb.ROUND_ROBIN
    assert kdb._mode(i, kdb.WIDEST_TIGHT) == kdb.WIDEST_TIGHT | kdb.COORDS_INT32
    # an explicit type wins over the dtype (uint32 data passed as an int32 view)
    assert kdb._mode(i, kdb.ROUND_ROBIN | kdb.COORDS_UINT32) == kdb.ROUND_ROBIN | kdb.COORDS_UINT32
    if getattr(torch, "uint32", None) is not None:
        u = i.view(torch.uint32)
        assert kdb._mode(u, kdb.ROUND_ROBIN) == kdb.ROUND_ROBIN | kdb.COORDS_UINT32


def test_tuning_file_parser_survives_mutated_input(lib, tmp_path):
    import random

    rng = random.Random(7)
    part = kdb.kdb_tuning_shapes(kdb.TUNE_PARTITION)
    rad = kdb.kdb_tuning_shapes(kdb.TUNE_RADIX)
    good = json.dumps({"partition": list(part[1]), "radix": list(rad[1]), "digit_bits": 6,
                       "table": [{"log2n": 20, "k": 3, "stride": 12, "mode": 0, "partition": list(part[0]),
                                  "radix": list(rad[1]), "digit_bits": 8}]}).encode()
    f = tmp_path / "t.json"
    try:
        for i in range(400):
            b = bytearray(good)
            for _ in range(rng.randint(1, 6)):
                op = rng.randrange(4)
                p = rng.randrange(len(b) + 1)
                if op == 0 and b:
                    del b[min(p, len(b) - 1)]
                elif op == 1:
                    b[p:p] = bytes([rng.randrange(256)])
                elif op == 2 and b:
                    b[min(p, len(b) - 1)] = rng.choice(b"0123456789,[]{}\": -+e\n\x00")
                else:
                    b = b[:p]
            if i % 50 == 0:
                b = bytes(rng.randrange(256) for _ in range(rng.randrange(2000)))
            f.write_bytes(bytes(b))
            rc = lib.kdb_load_tuning(str(f).encode())
            assert rc in (kdb.OK, kdb.ERR_INVALID_ARGUMENT)
            p_idx, r_idx, bits = kdb.kdb_get_tuning()
            assert 0 <= p_idx < len(part) and 0 <= r_idx < len(rad) and bits in (6, 8)
            (p_idx, r_idx, bits), _ = kdb.kdb_lookup_tuning(2**19, 3, 12)
            assert 0 <= p_idx < len(part) and 0 <= r_idx < len(rad) and bits in (6, 8)
    finally:
        kdb.kdb_clear_tuning_table()
        kdb.kdb_set_tuning(0, 0)


def test_binding_constants_match_the_header():
    """The binding's copies of the header's limits (the no-alloc build's point
    count and static workspace size) are the header's values."""
    import re

    text = open(kdb.HEADER).read()
    pts = int(re.search(r"#define KDB_NOALLOC_MAX_POINTS (\d+)", text).group(1))
    m = re.search(r"#define KDB_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", text)
    assert pts == kdb.NOALLOC_MAX_POINTS
    assert int(m.group(1)) << int(m.group(2)) == kdb.NOALLOC_SCRATCH_BYTES


def test_memory_mode_setting_and_lean_sizes(lib):
    """The memory-mode setting round trip, and the lean build's device memory:
    at most 40 B per point for float3 at 1e8 (against about 146 for the
    default), one tag and one index per point, a copy of the records and one
    subtree's workspace."""
    try:
        assert kdb.kdb_set_memory_mode(kdb.MEMORY_LEAN) == kdb.MEMORY_AUTO
        assert kdb.kdb_set_memory_mode(7) == kdb.MEMORY_LEAN  # refused: unchanged
        assert kdb.kdb_set_memory_mode(kdb.MEMORY_FAST) == kdb.MEMORY_LEAN
    finally:
        kdb.kdb_set_memory_mode(kdb.MEMORY_AUTO)
    n = 100_000_000
    lean = kdb.kdb_lean_workspace_size(n, 3, 12)
    fast = lib.kdb_workspace_size(n, 3, 12, kdb.ROUND_ROBIN)
    assert 4 * n + 12 * n + 4 * n < lean <= 40 * n < fast
    for k, stride, mode in [(3, 16, kdb.WIDEST_EXTENT), (3, 12, kdb.WIDEST_TIGHT), (1, 4, kdb.COORDS_INT32),
                            (4, 16, kdb.ROUND_ROBIN)]:
        b = kdb.kdb_lean_workspace_size(n, k, stride, mode)
        assert (8 + stride) * n < b <= (8 + stride + 24) * n, (k, stride, mode)
    assert kdb.kdb_lean_workspace_size(3, 3, 12) == 0  # too few points for a chosen level
    assert kdb.kdb_lean_workspace_size(4, 3, 12) > 0
    assert kdb.kdb_lean_workspace_size(n, 3, 12, kdb.WIDEST_EXTENT | kdb.COORDS_INT32) == 0
