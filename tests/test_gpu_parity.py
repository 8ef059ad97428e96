"""CUDA path against the CPU oracle, through the C ABI.

Every comparison is exact: the build only compares coordinates and moves
records, so the GPU output must equal the oracle's byte for byte (records and
original indices).  Sizes span many radix tiles (4096 items) with ragged
tails; the edge cases are the degenerate ones of the method (N <= 3, perfect
trees, all points equal, heavy ties, signed zeros, infinities, k = 1, payload
bytes, empty and one-point sets in a batch).
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth
from tests.golden_io import fig1, walkthrough

pytestmark = pytest.mark.gpu

RR, WIDEST = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT


def gpu_build(pts: np.ndarray, k: int, mode: int):
    d = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    orig = torch.empty(pts.shape[0], dtype=torch.int32, device="cuda")
    kdb.kdb_build_ex(d, k, mode, out_orig_index=orig)
    torch.cuda.synchronize()
    return d.cpu().numpy(), orig.cpu().numpy()


def assert_same(pts, k, mode):
    want, worig = oracle.build(pts, k, mode)
    got, gorig = gpu_build(pts, k, mode)
    if not np.array_equal(gorig, worig):
        bad = int(np.flatnonzero(gorig != worig)[0])
        raise AssertionError(f"N={len(pts)} k={k} mode={mode}: node {bad} holds {gorig[bad]}, "
                             f"oracle {worig[bad]}")
    assert got.view(np.uint32).tobytes() == want.view(np.uint32).tobytes()


def tie_grid(n, k, levels, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, levels, size=(n, k)).astype(np.float32)


@pytest.mark.parametrize("mode", [RR, WIDEST])
@pytest.mark.parametrize("n", [2, 3, 5, 10, 31, 32, 100, 1000, 4095, 4096, 4097, 12289, 65537,
                               300001])
def test_uniform_float3(n, mode):
    assert_same(synth.uniform(n, 3, seed=n), 3, mode)


@pytest.mark.parametrize("mode", [RR, WIDEST])
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_dimensions(k, mode):
    assert_same(synth.uniform(20011, k, seed=k), k, mode)


@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_mixed_with_duplicates(mode):
    assert_same(synth.mixed(200003, 3, seed=1), 3, mode)


@pytest.mark.parametrize("mode", [RR, WIDEST])
@pytest.mark.parametrize("levels", [1, 2, 3, 50])
def test_heavy_ties(levels, mode):
    assert_same(tie_grid(50000, 3, levels, seed=levels), 3, mode)


@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_signed_zero_and_infinities(mode):
    rng = np.random.default_rng(3)
    vals = np.array([-np.inf, -1.0, -0.0, 0.0, 1e-42, 1.0, np.inf], dtype=np.float32)
    pts = vals[rng.integers(0, len(vals), size=(30000, 3))]
    assert_same(pts, 3, mode)


@pytest.mark.parametrize("mode", [RR, WIDEST])
@pytest.mark.parametrize("stride_floats", [3, 4, 5, 8])
def test_payload_strides(stride_floats, mode):
    pts = synth.with_stride(synth.uniform(40000, 3, seed=9), stride_floats)
    assert_same(pts, 3, mode)


def test_perfect_trees():
    for m in [2, 3, 12, 13, 16]:
        assert_same(synth.uniform((1 << m) - 1, 3, seed=m), 3, RR)


def test_aniso_float4_widest():
    assert_same(synth.aniso_float4(100003, seed=2), 3, WIDEST)


def test_config1_uniform_1000():
    """N=1000 float3, uniform [0,1)^3, seed 0, round robin."""
    assert_same(synth.uniform(1000, 3, seed=0), 3, RR)


def test_paper_examples_on_gpu():
    pts, expected = fig1()
    got, _ = gpu_build(pts, 2, RR)
    np.testing.assert_array_equal(got, expected)
    blocks = walkthrough()
    _, _, _, x0, y0 = blocks[0]
    pts = np.array([x0, y0], dtype=np.float32).T.copy()
    got, _ = gpu_build(pts, 2, RR)
    _, _, _, xf, yf = blocks[-1]
    np.testing.assert_array_equal(got, np.array([xf, yf], dtype=np.float32).T)


def test_split_dims_output():
    pts = synth.uniform(5000, 3, seed=4)
    d = torch.from_numpy(pts).cuda()
    dims = torch.empty(5000, dtype=torch.uint8, device="cuda")
    kdb.kdb_build_ex(d, 3, RR, out_split_dim=dims)
    lv = np.floor(np.log2(np.arange(5000) + 1)).astype(np.int64)
    np.testing.assert_array_equal(dims.cpu().numpy(), lv % 3)


def test_user_workspace_and_repeatability():
    pts = synth.mixed(70001, 3, seed=8)
    want, _ = oracle.build(pts, 3, WIDEST)
    nbytes = kdb.kdb_workspace_size(70001, 3, 12, WIDEST)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        d = torch.from_numpy(pts).cuda()
        kdb.kdb_build_ex(d, 3, WIDEST, workspace=ws)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_host_buffer_entry_point():
    pts = synth.uniform(50000, 3, seed=12)
    want, _ = oracle.build(pts, 3, RR)
    h = torch.from_numpy(pts.copy()).pin_memory()
    kdb.kdb_build_host(h, 3, RR)
    assert np.array_equal(h.numpy(), want)


@pytest.mark.parametrize("path", ["mapped", "copied_pageable", "copied_payload"])
@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_host_buffer_paths(mode, path):
    """12M records (144-192 MB) in host memory.  Pinned records without payload
    are read and written in place by the kernels ("mapped"); pageable records,
    or records with payload, are copied to the device in two chunks overlapped
    with the first pass.  Every path gives the device build's tree, and a NaN
    leaves the host records as they were."""
    pts = synth.mixed(12_000_000, 3, seed=13)
    if path == "copied_payload":
        pts = synth.with_stride(pts, 4)
    d = torch.from_numpy(pts).cuda()
    kdb.kdb_build(d, 3, mode)

    def host(a):
        t = torch.from_numpy(a.copy())
        return t if path == "copied_pageable" else t.pin_memory()

    h = host(pts)
    kdb.kdb_build_host(h, 3, mode)
    assert torch.equal(h.view(torch.int32), d.cpu().view(torch.int32))
    bad = pts.copy()
    bad[11_999_000, 1] = np.nan  # in the last chunk
    hb = host(bad)
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build_host(hb, 3, mode)
    assert e.value.code == kdb.ERR_NAN_INPUT
    assert np.array_equal(hb.numpy().view(np.uint32), bad.view(np.uint32))


@pytest.mark.parametrize("n", [2, 3, 1000, 8191, 8192, 300001])
def test_host_buffer_mapped_small_and_ragged(n):
    pts = synth.uniform(n, 2, seed=n)
    want, _ = oracle.build(pts, 2, RR)
    h = torch.from_numpy(pts.copy()).pin_memory()
    kdb.kdb_build_host(h, 2, RR)
    assert np.array_equal(h.numpy().view(np.uint32), want.view(np.uint32))


def test_host_buffer_mapped_int32_and_tight():
    pts = synth.int32_uniform(400003, 1, seed=5)
    want, _ = oracle.build(pts, 1, RR)
    h = torch.from_numpy(pts.copy()).pin_memory()
    kdb.kdb_build_host(h, 1, RR)
    assert np.array_equal(h.numpy(), want)
    pts = synth.mixed(400003, 3, seed=6)
    want, _ = oracle.build(pts, 3, oracle.WIDEST_TIGHT)
    h = torch.from_numpy(pts.copy()).pin_memory()
    kdb.kdb_build_host(h, 3, kdb.WIDEST_TIGHT)
    assert np.array_equal(h.numpy().view(np.uint32), want.view(np.uint32))


def test_host_buffer_in_place_placement_copies():
    """Under the in-place placement setting the records go through a device
    copy (the mapped path needs the default placement); same tree."""
    pts = synth.uniform(200003, 3, seed=8)
    want, _ = oracle.build(pts, 3, RR)
    prev = kdb.kdb_set_placement(kdb.PLACEMENT_IN_PLACE)
    try:
        h = torch.from_numpy(pts.copy()).pin_memory()
        kdb.kdb_build_host(h, 3, RR)
    finally:
        kdb.kdb_set_placement(prev)
    assert np.array_equal(h.numpy().view(np.uint32), want.view(np.uint32))


def test_streams_run_independently():
    a = synth.uniform(100000, 3, seed=21)
    b = synth.mixed(100000, 3, seed=22)
    wa, _ = oracle.build(a, 3, RR)
    wb, _ = oracle.build(b, 3, WIDEST)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    kdb.kdb_build(da, 3, RR, stream=s1)
    kdb.kdb_build(db, 3, WIDEST, stream=s2)
    torch.cuda.synchronize()
    assert np.array_equal(da.cpu().numpy(), wa) and np.array_equal(db.cpu().numpy(), wb)


@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_batched_equals_each_set_alone(mode):
    sizes = [0, 1, 2, 3, 7, 100, 4097, 1, 0, 25000, 999, 65536, 5]
    sizes += [int(s) for s in synth.lognormal_sizes(40, 100, 20000, seed=3)]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = synth.mixed(int(offs[-1]), 3, seed=4)
    d = torch.from_numpy(pts).cuda()
    kdb.kdb_build_batched(d, offs.tolist(), 3, mode)
    got = d.cpu().numpy()
    for b in range(len(sizes)):
        lo, hi = offs[b], offs[b + 1]
        if hi - lo == 0:
            continue
        want, _ = oracle.build(pts[lo:hi], 3, mode)
        assert np.array_equal(got[lo:hi].view(np.uint32), want.view(np.uint32)), f"set {b}"


# ------------------------------------------------------------- validation --
@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_validate_accepts_trees_and_rejects_planted_errors(mode):
    pts = synth.uniform(30000, 3, seed=30)
    want, _ = oracle.build(pts, 3, mode)
    d = torch.from_numpy(want).cuda()
    assert kdb.kdb_validate(d, 3, mode) == -1
    bad = want.copy()
    bad[[5, 20000]] = bad[[20000, 5]]
    assert kdb.kdb_validate(torch.from_numpy(bad).cuda(), 3, mode) >= 0
    # the unbuilt input is not a tree
    assert kdb.kdb_validate(torch.from_numpy(pts).cuda(), 3, mode) >= 0


# ---------------------------------------------------------------- faults --
def test_nan_input_is_reported_and_records_untouched():
    pts = synth.uniform(10000, 3, seed=1)
    pts[777, 1] = np.nan
    d = torch.from_numpy(pts).cuda()
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build(d, 3, RR)
    assert e.value.code == kdb.ERR_NAN_INPUT
    assert np.array_equal(d.cpu().numpy().view(np.uint32), pts.view(np.uint32))


def test_allocation_failure_is_reported():
    pts = synth.uniform(10000, 3, seed=2)
    d = torch.from_numpy(pts).cuda()
    kdb.kdb_debug_inject_fault(kdb.FAULT_ALLOC, 0)
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build(d, 3, RR)
    assert e.value.code == kdb.ERR_OUT_OF_MEMORY
    assert np.array_equal(d.cpu().numpy(), pts)


def test_lookback_wait_runs_out_and_context_stays_usable():
    """The radix passes wait on a look-back value no block ever writes: every
    bounded wait gives up after ~200 us, the build reports a timeout, leaves
    the records alone, and the next build works."""
    pts = synth.uniform(3 * 4096 + 5, 3, seed=3)
    d = torch.from_numpy(pts).cuda()
    kdb.kdb_debug_inject_fault(kdb.FAULT_LOOKBACK, 200)
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build(d, 3, RR)
    assert e.value.code == kdb.ERR_TIMEOUT
    assert np.array_equal(d.cpu().numpy(), pts)
    assert_same(pts, 3, RR)


@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_batched_large_sets_use_segmented_levels(mode):
    """All sets long enough that the top levels sort segment by segment."""
    sizes = [20000, 16383, 70001, 40000, 16384, 131071]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = synth.uniform(int(offs[-1]), 3, seed=8)
    d = torch.from_numpy(pts).cuda()
    kdb.kdb_build_batched(d, offs.tolist(), 3, mode)
    got = d.cpu().numpy()
    for b in range(len(sizes)):
        lo, hi = offs[b], offs[b + 1]
        want, _ = oracle.build(pts[lo:hi], 3, mode)
        assert np.array_equal(got[lo:hi].view(np.uint32), want.view(np.uint32)), f"set {b}"


@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_large_single_builds_exact(mode):
    """2^21 + 3 points: 9 segmented levels then the packed-key levels."""
    assert_same(synth.mixed((1 << 21) + 3, 3, seed=77), 3, mode)


# -------------------------------------------------------------- placement --
PLACEMENT_CASES = {
    # name: (points, k, mode); record widths on both sides of the spare
    # workspace the gather placement needs
    "float3_rr": (lambda: synth.uniform(300001, 3, seed=51), 3, RR),
    "float4_widest": (lambda: synth.aniso_float4(200003, seed=52), 3, WIDEST),
    "stride8_rr": (lambda: synth.with_stride(synth.uniform(70001, 3, seed=53), 8), 3, RR),
    "stride40_widest": (lambda: synth.with_stride(synth.uniform(50001, 3, seed=54), 40), 3, WIDEST),
    "k4_rr": (lambda: synth.uniform(90001, 4, seed=55), 4, RR),
    "k1_small": (lambda: synth.uniform(5000, 1, seed=56), 1, RR),
}


@pytest.mark.parametrize("placement", [kdb.PLACEMENT_AUTO, kdb.PLACEMENT_IN_PLACE])
@pytest.mark.parametrize("case", sorted(PLACEMENT_CASES))
def test_placement_modes_agree_with_oracle(case, placement):
    gen, k, mode = PLACEMENT_CASES[case]
    prev = kdb.kdb_set_placement(placement)
    try:
        assert_same(gen(), k, mode)
    finally:
        kdb.kdb_set_placement(prev)


@pytest.mark.parametrize("placement", [kdb.PLACEMENT_AUTO, kdb.PLACEMENT_IN_PLACE])
def test_placement_modes_batched(placement):
    sizes = [3, 70001, 0, 5000, 16384, 1, 40000]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = synth.mixed(int(offs[-1]), 3, seed=57)
    prev = kdb.kdb_set_placement(placement)
    try:
        d = torch.from_numpy(pts).cuda()
        kdb.kdb_build_batched(d, offs.tolist(), 3, RR)
        got = d.cpu().numpy()
    finally:
        kdb.kdb_set_placement(prev)
    for b in range(len(sizes)):
        lo, hi = offs[b], offs[b + 1]
        if hi > lo:
            want, _ = oracle.build(pts[lo:hi], 3, RR)
            assert np.array_equal(got[lo:hi].view(np.uint32), want.view(np.uint32)), f"set {b}"


@pytest.mark.parametrize("placement", [kdb.PLACEMENT_AUTO, kdb.PLACEMENT_IN_PLACE])
def test_failure_after_first_pivots_leaves_records_untouched(placement):
    """A partition pass times out after the root's record was already written
    at its node (records without payload go straight to their nodes): the
    build reports the timeout, the caller's array is exactly the input again,
    and the next build works."""
    pts = synth.uniform(100003, 3, seed=61)
    d = torch.from_numpy(pts).cuda()
    prev = kdb.kdb_set_placement(placement)
    try:
        kdb.kdb_debug_inject_fault(kdb.FAULT_LOOKBACK_PARTITION, 200)
        with pytest.raises(kdb.KdbError) as e:
            kdb.kdb_build(d, 3, RR)
        assert e.value.code == kdb.ERR_TIMEOUT
        assert np.array_equal(d.cpu().numpy().view(np.uint32), pts.view(np.uint32))
        assert_same(pts, 3, RR)
    finally:
        kdb.kdb_set_placement(prev)


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("n", [16383, 16384, 24575, 32767, 32768, 49153, 131071, 131072])
def test_level1_list_from_its_last_pass(n, k):
    """Round robin over one set with at least two global levels: the list of
    the level-1 dimension leaves its last digit pass already on level 1
    (sorted by side of the root, then key), the root dropped.  Sizes around
    the first ones with two global levels, perfect trees and ragged ones,
    ties in the root's dimension (the side of equal keys is decided by
    index)."""
    pts = synth.uniform(n, k, seed=n + k)
    pts[::3, 0] = pts[7, 0]  # a third of the points share the root dimension's key
    assert_same(pts, k, RR)
    ints = synth.int32_uniform(n, k, seed=n)
    ints[::5, 0] = -1
    assert_same(ints, k, RR)
