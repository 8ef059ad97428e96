"""kdb_build_noalloc: the build for callers that cannot allocate device memory
when they build (a device-memory budget fixed at start-up, or loops where an
allocation must not fail or stall).  Its workspace is one static device array
inside the library; it must give exactly what kdb_build gives, call after
call, even though each call finds the previous call's leftovers in that array.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest
import torch

from paper_2211_00120_gb300 import kdb, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_kdb_build_on_two_calls_in_a_row():
    cases = [
        (synth.mixed(100003, 3, seed=41), 3, kdb.ROUND_ROBIN),
        (synth.aniso_float4(kdb.NOALLOC_MAX_POINTS, seed=42), 3, kdb.WIDEST_EXTENT),
    ]
    for pts, k, mode in cases:  # two calls back to back, different sizes and modes
        ref = torch.from_numpy(pts).cuda()
        kdb.kdb_build(ref, k, mode)
        got = torch.from_numpy(pts).cuda()
        kdb.kdb_build_noalloc(got, k, mode)
        torch.cuda.synchronize()
        # bit-exact, the tolerance of every parity test here
        assert np.array_equal(got.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))


def test_noalloc_rejects_sizes_beyond_its_limit():
    pts = torch.zeros((kdb.NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build_noalloc(pts, 3, kdb.ROUND_ROBIN)
    assert e.value.code == kdb.ERR_INVALID_ARGUMENT
    # within the point limit but a workspace larger than the static array:
    # 8 KiB records make the placement's staging area alone 64 MiB
    wide = torch.zeros((kdb.NOALLOC_MAX_POINTS, 2048), dtype=torch.float32, device="cuda")
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build_noalloc(wide, 3, kdb.WIDEST_EXTENT)
    assert e.value.code == kdb.ERR_INVALID_ARGUMENT
