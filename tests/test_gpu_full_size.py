"""CUDA path at the full workload sizes, in the launch configuration the
benchmark times (kdb_build on a device-resident array, library workspace).

  - 1e7 float3, half uniform / half 64 Gaussian clusters with 1% exact
    duplicates, round robin: compared array for array with the whole oracle
    build (about half a minute of CPU).
  - 1e8 float3 uniform, round robin, and 1e8 float4 in the anisotropic box
    [0,100)x[0,1)x[0,10) with the original index as payload, widest extent:
    the oracle's full build would take minutes, so the oracle's invariant
    checker runs on the whole output instead -- the records are a permutation
    of the input and every node satisfies the strict k-d condition against
    every ancestor, with the widest dimensions recomputed top-down.  Under the
    strict (coordinate, original index) order the valid arrangement is unique,
    so this is equality with the oracle; a few nodes are also selected
    directly by the oracle along their root paths (Observation 1).
Every comparison is exact.
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth

pytestmark = pytest.mark.gpu

RR, WIDEST, TIGHT = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT, kdb.WIDEST_TIGHT


def build_like_bench(pts: np.ndarray, k: int, mode: int):
    """kdb_build exactly as timed, plus kdb_build_ex for the original indices;
    both must give the same records."""
    src = torch.from_numpy(pts).cuda()
    work = src.clone()
    kdb.kdb_build(work, k, mode)
    ex = src.clone()
    orig = torch.empty(pts.shape[0], dtype=torch.int32, device="cuda")
    kdb.kdb_build_ex(ex, k, mode, out_orig_index=orig)
    torch.cuda.synchronize()
    assert torch.equal(work.view(torch.int32), ex.view(torch.int32))
    out = work.cpu().numpy()
    del src, work, ex
    return out, orig.cpu().numpy()


def sampled_nodes(n: int):
    return [0, 1, 2, n // 2 - 1, n - 1]


def test_mixed_1e7_round_robin_equals_oracle():
    pts = synth.mixed(10_000_000, 3, seed=1)
    got, gorig = build_like_bench(pts, 3, RR)
    want, worig = oracle.build(pts, 3, RR)
    if not np.array_equal(gorig, worig):
        bad = int(np.flatnonzero(gorig != worig)[0])
        raise AssertionError(f"node {bad} holds {gorig[bad]}, oracle {worig[bad]}")
    assert got.view(np.uint32).tobytes() == want.view(np.uint32).tobytes()


def test_mixed_1e7_tight_box_equals_oracle():
    pts = synth.mixed(10_000_000, 3, seed=1)
    got, gorig = build_like_bench(pts, 3, TIGHT)
    want, worig = oracle.build(pts, 3, TIGHT)
    if not np.array_equal(gorig, worig):
        bad = int(np.flatnonzero(gorig != worig)[0])
        raise AssertionError(f"node {bad} holds {gorig[bad]}, oracle {worig[bad]}")
    assert got.view(np.uint32).tobytes() == want.view(np.uint32).tobytes()


def test_uniform_1e8_float3_round_robin():
    pts = synth.uniform(100_000_000, 3, seed=0)
    got, gorig = build_like_bench(pts, 3, RR)
    assert oracle.check(pts, got, gorig, 3, RR) == -1
    for s in sampled_nodes(len(pts))[:3]:
        assert gorig[s] == oracle.node(pts, 3, RR, s)


def test_aniso_1e8_float4_widest():
    pts = synth.aniso_float4(100_000_000, seed=2)
    got, gorig = build_like_bench(pts, 3, WIDEST)
    # the payload is the original index, moved with its record
    assert np.array_equal(got[:, 3].view(np.uint32), gorig.view(np.uint32))
    assert oracle.check(pts, got, gorig, 3, WIDEST) == -1
    for s in sampled_nodes(len(pts))[:3]:
        assert gorig[s] == oracle.node(pts, 3, WIDEST, s)
