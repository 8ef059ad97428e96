"""uint32 coordinates (KDB_COORDS_UINT32) on the CUDA path, against the CPU
oracle through the C ABI.  Exact comparisons.  Records travel as int32 views
with the flag given explicitly, so that no torch uint32 kernels are needed;
one test goes through a torch uint32 tensor and the binding's dtype rule."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb

pytestmark = pytest.mark.gpu

RR, WIDEST, TIGHT = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT, kdb.WIDEST_TIGHT
U = kdb.COORDS_UINT32
EDGE = np.array([0, 1, 2**24, 2**24 + 1, 2**31 - 1, 2**31, 2**31 + 1, 2**32 - 2, 2**32 - 1],
                dtype=np.uint64)


def full_range(n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**32, size=(n, k), dtype=np.uint64).astype(np.uint32)


def gpu_build(pts, k, mode):
    d = torch.from_numpy(np.ascontiguousarray(pts).view(np.int32)).cuda()
    orig = torch.empty(pts.shape[0], dtype=torch.int32, device="cuda")
    kdb.kdb_build_ex(d, k, mode | U, out_orig_index=orig)
    torch.cuda.synchronize()
    return d.cpu().numpy().view(np.uint32), orig.cpu().numpy()


def assert_same(pts, k, mode):
    want, worig = oracle.build(pts, k, mode)
    got, gorig = gpu_build(pts, k, mode)
    if not np.array_equal(gorig, worig):
        bad = int(np.flatnonzero(gorig != worig)[0])
        raise AssertionError(f"N={len(pts)} k={k} mode={mode}: node {bad} holds {gorig[bad]}, "
                             f"oracle {worig[bad]}")
    assert got.tobytes() == want.tobytes()


@pytest.mark.parametrize("mode", [RR, TIGHT])
@pytest.mark.parametrize("n", [2, 3, 1000, 4097, 8192, 65537, 300001])
def test_full_range_uint3(n, mode):
    assert_same(full_range(n, 3, seed=n), 3, mode)


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_values_on_both_sides_of_the_sign_bit(mode):
    rng = np.random.default_rng(5)
    pts = EDGE[rng.integers(0, len(EDGE), size=(40000, 3))].astype(np.uint32)
    assert_same(pts, 3, mode)


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_dimensions_round_robin(k):
    # k >= 4 runs the rank-sort path
    assert_same(full_range(20011, k, seed=k), k, RR)


def test_heavy_ties_small_range():
    rng = np.random.default_rng(2)
    pts = rng.integers(0, 6, size=(50000, 3)).astype(np.uint32)
    for mode in (RR, TIGHT):
        assert_same(pts, 3, mode)


def test_tight_root_uses_unsigned_extents():
    # x spans 2^31 + 5 and y 2^31 unsigned, so the root splits in x (as int32
    # the y side would be wider)
    pts = np.array([[0, 0], [2**31 + 5, 1], [1, 2**31]], dtype=np.uint32)
    got, orig = gpu_build(pts, 2, TIGHT)
    assert list(orig) == [2, 0, 1]


def test_batched_sets_and_validator():
    sizes = [1, 5000, 0, 70001, 3]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = full_range(int(offs[-1]), 3, seed=21)
    for mode in (RR, TIGHT):
        d = torch.from_numpy(pts.view(np.int32)).cuda()
        kdb.kdb_build_batched(d, offs.tolist(), 3, mode | U)
        got = d.cpu().numpy().view(np.uint32)
        for b in range(len(sizes)):
            lo, hi = offs[b], offs[b + 1]
            if hi > lo:
                want = oracle.build(pts[lo:hi], 3, mode)[0]
                assert np.array_equal(got[lo:hi], want), (mode, b)
                w = torch.from_numpy(want.view(np.int32)).cuda()
                assert kdb.kdb_validate(w, 3, mode | U) == -1
        # the unsigned order, not the signed order of the bits, decides validity
        tree = got[offs[3]:offs[4]].copy()
        assert kdb.kdb_validate(torch.from_numpy(tree.view(np.int32)).cuda(), 3, mode | U) == -1
        tree[[1, 2]] = tree[[2, 1]]
        assert kdb.kdb_validate(torch.from_numpy(tree.view(np.int32)).cuda(), 3, mode | U) >= 0


def test_host_buffer_mapped():
    pts = full_range(200003, 3, seed=4)
    want, _ = oracle.build(pts, 3, RR)
    h = torch.from_numpy(pts.view(np.int32).copy()).pin_memory()
    kdb.kdb_build_host(h, 3, RR | U)
    assert np.array_equal(h.numpy().view(np.uint32), want)


def test_refusals():
    d = torch.from_numpy(full_range(1000, 3, seed=1).view(np.int32)).cuda()
    for mode in (WIDEST | U, RR | U | kdb.COORDS_INT32):
        with pytest.raises(kdb.KdbError) as e:
            kdb.kdb_build(d, 3, mode)
        assert e.value.code == kdb.ERR_INVALID_ARGUMENT


def test_torch_uint32_tensor_sets_the_flag():
    if getattr(torch, "uint32", None) is None:
        pytest.skip("this torch has no uint32 dtype")
    pts = full_range(30011, 2, seed=9)
    want, _ = oracle.build(pts, 2, RR)
    d = torch.from_numpy(pts.view(np.int32)).cuda().view(torch.uint32)
    kdb.kdb_build(d, 2, RR)
    assert np.array_equal(d.view(torch.int32).cpu().numpy().view(np.uint32), want)
