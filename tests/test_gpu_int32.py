"""int32 coordinates (KDB_COORDS_INT32; the paper's int1 / int2 data) on the
CUDA path, against the CPU oracle through the C ABI.  Exact comparisons."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth
from tests.golden_io import walkthrough
from tests.test_gpu_parity import assert_same, gpu_build

pytestmark = pytest.mark.gpu

RR, WIDEST, TIGHT = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT, kdb.WIDEST_TIGHT
EDGE = np.array([-2**31, -2**31 + 1, -1, 0, 1, 2**24, 2**24 + 1, 2**31 - 2, 2**31 - 1],
                dtype=np.int64)


def full_range(n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-2**31, 2**31, size=(n, k), dtype=np.int64).astype(np.int32)


@pytest.mark.parametrize("mode", [RR, TIGHT])
@pytest.mark.parametrize("n", [2, 3, 1000, 4097, 8192, 65537, 300001])
def test_full_range_int3(n, mode):
    assert_same(full_range(n, 3, seed=n), 3, mode)


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_extremes_and_float_colliding_pairs(mode):
    rng = np.random.default_rng(5)
    pts = EDGE[rng.integers(0, len(EDGE), size=(40000, 3))].astype(np.int32)
    assert_same(pts, 3, mode)


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_dimensions_round_robin(k):
    # k = 1 is Table 1's int1; k >= 4 runs the rank-sort path
    assert_same(full_range(20011, k, seed=k), k, RR)


def test_heavy_ties_small_range():
    rng = np.random.default_rng(2)
    pts = rng.integers(-3, 3, size=(50000, 3)).astype(np.int32)
    for mode in (RR, TIGHT):
        assert_same(pts, 3, mode)


def test_nan_bit_patterns_are_ordinary_integers():
    pts = full_range(5000, 3, seed=3)
    pts[::7, 1] = np.int32(0x7FC00000)  # a quiet NaN's bits, as an integer
    assert_same(pts, 3, RR)


@pytest.mark.parametrize("stride_ints", [3, 4, 6])
def test_payload_strides(stride_ints):
    base = full_range(30000, 3, seed=11)
    rng = np.random.default_rng(12)
    pts = np.concatenate([base, rng.integers(-2**31, 2**31, size=(30000, stride_ints - 3),
                                             dtype=np.int64).astype(np.int32)], axis=1)
    for mode in (RR, TIGHT):
        assert_same(np.ascontiguousarray(pts), 3, mode)


def test_sec5_walkthrough_int2_on_gpu():
    blocks = walkthrough()
    _, _, _, x0, y0 = blocks[0]
    pts = np.array([x0, y0], dtype=np.int32).T.copy()
    got, _ = gpu_build(pts, 2, RR)
    _, _, _, xf, yf = blocks[-1]
    np.testing.assert_array_equal(got, np.array([xf, yf], dtype=np.int32).T)


def test_batched_int_sets_and_validator():
    sizes = [1, 5000, 0, 70001, 3]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = full_range(int(offs[-1]), 3, seed=21)
    for mode in (RR, TIGHT):
        d = torch.from_numpy(pts).cuda()
        kdb.kdb_build_batched(d, offs.tolist(), 3, mode)
        got = d.cpu().numpy()
        for b in range(len(sizes)):
            lo, hi = offs[b], offs[b + 1]
            if hi > lo:
                want = oracle.build(pts[lo:hi], 3, mode)[0]
                assert np.array_equal(got[lo:hi], want), (mode, b)
                assert kdb.kdb_validate(torch.from_numpy(want).cuda(), 3, mode) == -1
        # the int order, not the float order of the bits, decides validity
        bad = got[offs[3]:offs[4]].copy()
        bad[[1, 2]] = bad[[2, 1]]
        assert kdb.kdb_validate(torch.from_numpy(bad).cuda(), 3, mode) >= 0


def test_clipped_domain_rule_refuses_int32():
    d = torch.from_numpy(full_range(1000, 3, seed=1)).cuda()
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build(d, 3, WIDEST)
    assert e.value.code == kdb.ERR_INVALID_ARGUMENT
