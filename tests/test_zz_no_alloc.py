"""kdb_build_noalloc: the build for callers that cannot allocate device memory
when they build (a device-memory budget fixed at start-up, or loops where an
allocation must not fail or stall).  Its workspace is one static device array
inside the library, so every call finds the previous call's leftovers there.
Each call must still give exactly the oracle's tree (Sec. 2, Observation 1),
and exactly what kdb_build gives.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth

pytestmark = pytest.mark.gpu

RR, WIDEST, TIGHT = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT, kdb.WIDEST_TIGHT


def noalloc_equals_oracle(pts: np.ndarray, k: int, mode: int, what: str) -> None:
    got = torch.from_numpy(pts).cuda()
    kdb.kdb_build_noalloc(got, k, mode)
    torch.cuda.synchronize()
    out = got.cpu().numpy()
    want, _ = oracle.build(pts, k, mode)
    # bit-exact, the tolerance of every parity test here
    if not np.array_equal(out.view(np.uint32), want.view(np.uint32)):
        bad = int(np.flatnonzero((out.view(np.uint32) != want.view(np.uint32)).any(axis=1))[0])
        raise AssertionError(f"{what}: node {bad} differs from the oracle")
    ref = torch.from_numpy(pts).cuda()
    kdb.kdb_build(ref, k, mode)
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), what


def test_noalloc_matches_oracle_on_two_calls_in_a_row():
    cases = [
        (synth.mixed(100003, 3, seed=41), 3, RR),
        (synth.aniso_float4(kdb.NOALLOC_MAX_POINTS, seed=42), 3, WIDEST),
    ]
    for i, (pts, k, mode) in enumerate(cases):  # two calls back to back, different sizes and modes
        noalloc_equals_oracle(pts, k, mode, f"call {i}")


def test_noalloc_sequence_of_shapes_reuses_the_array():
    """Larger then smaller, repeated shapes, k = 3 (presorted lists) and k = 5
    (rank sorts), all three split rules and int32 coordinates, back to back:
    any region of the static array that a call expects zeroed and does not
    clear would show up in a later call."""
    cases = [
        (synth.uniform(kdb.NOALLOC_MAX_POINTS, 3, seed=50), 3, RR),
        (synth.mixed(9001, 3, seed=51), 3, TIGHT),
        (synth.mixed(9001, 3, seed=51), 3, TIGHT),
        (synth.mixed(200_000, 5, seed=52), 5, WIDEST),
        (synth.uniform(777, 5, seed=53), 5, RR),
        (synth.int32_uniform(150_000, 3, seed=54), 3, TIGHT | kdb.COORDS_INT32),
        (synth.mixed(33, 3, seed=55), 3, WIDEST),
        (synth.mixed(131_071, 3, seed=56), 3, RR),
        (synth.mixed(131_071, 3, seed=56), 3, RR),
    ]
    for i, (pts, k, mode) in enumerate(cases):
        noalloc_equals_oracle(pts, k, mode, f"call {i}")


def test_noalloc_workspace_just_below_the_limit():
    """A shape whose workspace is within a few KiB of the static array builds
    correctly (the array's end is used); the next stride up is refused."""
    n, k, mode = kdb.NOALLOC_MAX_POINTS, 3, WIDEST
    stride = 4 * k
    while kdb.kdb_workspace_size(n, k, stride + 4, mode) <= kdb.NOALLOC_SCRATCH_BYTES:
        stride += 4
    assert kdb.NOALLOC_SCRATCH_BYTES - kdb.kdb_workspace_size(n, k, stride, mode) < 64 << 10
    pts = synth.with_stride(synth.uniform(n, k, seed=60), stride // 4)
    noalloc_equals_oracle(pts, k, mode, f"stride {stride}")
    del pts
    wider = torch.zeros((n, stride // 4 + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build_noalloc(wider, k, mode)
    assert e.value.code == kdb.ERR_INVALID_ARGUMENT


def test_noalloc_rejects_sizes_beyond_its_limit():
    pts = torch.zeros((kdb.NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build_noalloc(pts, 3, RR)
    assert e.value.code == kdb.ERR_INVALID_ARGUMENT
    # within the point limit but a workspace larger than the static array:
    # 8 KiB records make the placement's staging area alone 64 MiB
    wide = torch.zeros((kdb.NOALLOC_MAX_POINTS, 2048), dtype=torch.float32, device="cuda")
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build_noalloc(wide, 3, WIDEST)
    assert e.value.code == kdb.ERR_INVALID_ARGUMENT
