"""The tight-bounding-box split rule (KDB_SPLIT_WIDEST_TIGHT) on the CUDA
path, against the CPU oracle, through the C ABI.  Exact comparisons, as for
the other rules: the build compares keys and moves records, and the extents
that pick a dimension are one float32 subtraction on each side."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth
from tests.golden_io import tight_box
from tests.test_gpu_parity import assert_same, gpu_build, tie_grid

pytestmark = pytest.mark.gpu

TIGHT = kdb.WIDEST_TIGHT
assert TIGHT == oracle.WIDEST_TIGHT


@pytest.mark.parametrize("n", [2, 3, 5, 10, 31, 100, 1000, 4095, 4096, 8191, 8192, 12289, 65537,
                               300001])
def test_uniform_float3(n):
    assert_same(synth.uniform(n, 3, seed=n), 3, TIGHT)


@pytest.mark.parametrize("k", [1, 2])
def test_fewer_dimensions(k):
    assert_same(synth.uniform(20011, k, seed=k), k, TIGHT)


def test_more_than_three_dimensions_are_refused():
    d = torch.from_numpy(synth.uniform(1000, 4, seed=1)).cuda()
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build(d, 4, TIGHT)
    assert e.value.code == kdb.ERR_INVALID_ARGUMENT


def test_mixed_clusters_and_duplicates():
    assert_same(synth.mixed(200003, 3, seed=1), 3, TIGHT)


@pytest.mark.parametrize("levels", [1, 2, 3, 50])
def test_heavy_ties(levels):
    assert_same(tie_grid(50000, 3, levels, seed=levels), 3, TIGHT)


def test_signed_zero_and_infinities():
    # boxes with an infinite side, and extents inf - inf = NaN
    rng = np.random.default_rng(3)
    vals = np.array([-np.inf, -1.0, -0.0, 0.0, 1e-42, 1.0, np.inf], dtype=np.float32)
    pts = vals[rng.integers(0, len(vals), size=(30000, 3))]
    assert_same(pts, 3, TIGHT)


@pytest.mark.parametrize("stride_floats", [3, 4, 5, 8])
def test_payload_strides(stride_floats):
    pts = synth.with_stride(synth.uniform(40000, 3, seed=9), stride_floats)
    assert_same(pts, 3, TIGHT)


def test_aniso_float4():
    assert_same(synth.aniso_float4(100003, seed=2), 3, TIGHT)


def test_hand_example_and_validator():
    pts, want, want_clipped = tight_box()
    got, _ = gpu_build(pts, 2, TIGHT)
    np.testing.assert_array_equal(got, want)
    assert kdb.kdb_validate(torch.from_numpy(want).cuda(), 2, TIGHT) == -1
    # the clipped-domain tree is not a tight-box tree, and the other way round
    assert kdb.kdb_validate(torch.from_numpy(want_clipped).cuda(), 2, TIGHT) >= 0
    assert kdb.kdb_validate(torch.from_numpy(want).cuda(), 2, kdb.WIDEST_EXTENT) >= 0


def test_split_dims_output_matches_the_oracle_checker():
    pts = synth.mixed(50000, 3, seed=12)
    d = torch.from_numpy(pts).cuda()
    dims = torch.empty(50000, dtype=torch.uint8, device="cuda")
    orig = torch.empty(50000, dtype=torch.int32, device="cuda")
    kdb.kdb_build_ex(d, 3, TIGHT, out_orig_index=orig, out_split_dim=dims)
    out = d.cpu().numpy()
    assert oracle.check(pts, out, orig.cpu().numpy(), 3, TIGHT) == -1
    # every node's dimension is the widest side of its subtree's box
    n = len(out)
    lo, hi = out.copy(), out.copy()
    for i in range(n - 1, -1, -1):
        for c in (2 * i + 1, 2 * i + 2):
            if c < n:
                lo[i] = np.minimum(lo[i], lo[c])
                hi[i] = np.maximum(hi[i], hi[c])
    ext = (hi - lo).astype(np.float32)
    want = np.zeros(n, np.int64)
    best = ext[:, 0].copy()
    for dd in (1, 2):
        better = ext[:, dd] > best
        want[better] = dd
        best[better] = ext[better, dd]
    np.testing.assert_array_equal(dims.cpu().numpy(), want)
    assert kdb.kdb_validate(d, 3, TIGHT) == -1


def test_batched_equals_each_set_alone_and_the_oracle():
    sizes = [0, 1, 2, 7, 8191, 8192, 30000, 5, 100003]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = synth.mixed(int(offs[-1]), 3, seed=21)
    d = torch.from_numpy(pts).cuda()
    kdb.kdb_build_batched(d, offs.tolist(), 3, TIGHT)
    got = d.cpu().numpy()
    for b in range(len(sizes)):
        lo, hi = offs[b], offs[b + 1]
        if hi - lo == 0:
            continue
        want = oracle.build(pts[lo:hi], 3, TIGHT)[0]
        assert got[lo:hi].view(np.uint32).tobytes() == want.view(np.uint32).tobytes(), b
