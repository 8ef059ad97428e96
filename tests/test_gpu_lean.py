"""The memory-lean build (kdb_set_memory_mode(MEMORY_LEAN)): the top four
levels by a radix select over the whole array, one move of every point to its
level-4 subtree, each subtree built alone.  Its tree must be the oracle's,
bit for bit, in every split rule and coordinate type; a NaN leaves the
records untouched."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth
from tests.test_gpu_parity import tie_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def lean_mode():
    prev = kdb.kdb_set_memory_mode(kdb.MEMORY_LEAN)
    yield
    kdb.kdb_set_memory_mode(prev)


def lean_build(pts, k, mode):
    d = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    kdb.kdb_build(d, k, mode)
    return d.cpu().numpy()


def check(pts, k, mode):
    got = lean_build(pts, k, mode)
    want, _ = oracle.build(pts, k, mode & 0xFF)
    if got.view(np.uint32).tobytes() != want.view(np.uint32).tobytes():
        bad = int(np.flatnonzero((got.view(np.uint32) != want.view(np.uint32)).any(axis=1))[0])
        raise AssertionError(f"node {bad}: {got[bad]} against the oracle's {want[bad]}")


CASES = [
    # (name, points, k, mode): several subtree sizes, ties, payload, types
    ("uniform3_rr", lambda: synth.uniform(300_001, 3, seed=41), 3, kdb.ROUND_ROBIN),
    ("mixed3_rr", lambda: synth.mixed(200_003, 3, seed=42), 3, kdb.ROUND_ROBIN),
    ("ties3_tight", lambda: tie_grid(150_001, 3, 5, seed=43), 3, kdb.WIDEST_TIGHT),
    ("aniso4_widest", lambda: synth.aniso_float4(250_007, seed=44), 3, kdb.WIDEST_EXTENT),
    ("aniso4_tight", lambda: synth.aniso_float4(99_991, seed=45), 3, kdb.WIDEST_TIGHT),
    ("mixed2_widest", lambda: synth.mixed(65_537, 2, seed=46), 2, kdb.WIDEST_EXTENT),
    ("uniform1_rr", lambda: synth.uniform(40_000, 1, seed=47), 1, kdb.ROUND_ROBIN),
    ("uniform4_rr", lambda: synth.uniform(120_000, 4, seed=48), 4, kdb.ROUND_ROBIN),
    ("small", lambda: synth.uniform(37, 3, seed=49), 3, kdb.ROUND_ROBIN),
    ("smallest", lambda: synth.uniform(4, 2, seed=50), 2, kdb.WIDEST_EXTENT),
]


@pytest.mark.parametrize("name,gen,k,mode", CASES, ids=[c[0] for c in CASES])
def test_lean_build_equals_oracle(name, gen, k, mode):
    check(gen(), k, mode)


def test_lean_build_integer_coordinates():
    pts = synth.int32_uniform(180_001, 3, seed=51)
    pts[::9, 2] = -3  # ties in one dimension
    check(pts, 3, kdb.WIDEST_TIGHT | kdb.COORDS_INT32)
    check(pts, 3, kdb.ROUND_ROBIN | kdb.COORDS_INT32)
    u = synth.int32_uniform(90_000, 2, seed=52).view(np.uint32)
    got = torch.from_numpy(u.view(np.int32).copy()).cuda()
    kdb.kdb_build(got, 2, kdb.ROUND_ROBIN | kdb.COORDS_UINT32)
    want, _ = oracle.build(u, 2, oracle.ROUND_ROBIN)
    assert got.cpu().numpy().view(np.uint32).tobytes() == want.view(np.uint32).tobytes()


def test_lean_and_default_builds_agree_at_2e6():
    pts = synth.uniform(2_000_000, 3, seed=53)
    lean = lean_build(pts, 3, kdb.ROUND_ROBIN)
    kdb.kdb_set_memory_mode(kdb.MEMORY_FAST)
    fast = lean_build(pts, 3, kdb.ROUND_ROBIN)
    assert lean.view(np.uint32).tobytes() == fast.view(np.uint32).tobytes()
    d = torch.from_numpy(lean).cuda()
    assert kdb.kdb_validate(d, 3, kdb.ROUND_ROBIN) == -1
    # a few nodes against the oracle's own computation of them
    for node in (0, 1, 2, 14, 15, 30, 1_000_000, 1_999_999):
        want = pts[oracle.node(pts, 3, oracle.ROUND_ROBIN, node)]
        assert lean[node].view(np.uint32).tolist() == want.view(np.uint32).tolist()


def test_lean_build_refuses_nan_and_leaves_records_untouched():
    pts = synth.uniform(100_000, 3, seed=54)
    pts[77_777, 1] = np.nan
    d = torch.from_numpy(pts.copy()).cuda()
    with pytest.raises(kdb.KdbError) as e:
        kdb.kdb_build(d, 3, kdb.ROUND_ROBIN)
    assert e.value.code == kdb.ERR_NAN_INPUT
    assert d.cpu().numpy().view(np.uint32).tobytes() == pts.view(np.uint32).tobytes()
    # the next build works
    ok = synth.uniform(100_000, 3, seed=55)
    check(ok, 3, kdb.ROUND_ROBIN)


def test_lean_workspace_is_small():
    """The lean build's device memory against the default's, per point."""
    n = 100_000_000
    lean = kdb.kdb_lean_workspace_size(n, 3, 12)
    fast = kdb.load().kdb_workspace_size(n, 3, 12, kdb.ROUND_ROBIN)
    assert lean / n <= 40 and fast / lean > 4


def test_automatic_mode_goes_lean_when_memory_is_short():
    """MEMORY_AUTO takes the lean build when the default workspace does not
    fit the free memory (made short here by the host-side test hook), the
    default build otherwise; both give the oracle's tree."""
    kdb.kdb_set_memory_mode(kdb.MEMORY_AUTO)
    pts = synth.uniform(400_000, 3, seed=56)
    want, _ = oracle.build(pts, 3, oracle.ROUND_ROBIN)
    lean_bytes = kdb.kdb_lean_workspace_size(len(pts), 3, 12)
    fast_bytes = kdb.load().kdb_workspace_size(len(pts), 3, 12, kdb.ROUND_ROBIN)
    assert lean_bytes < fast_bytes
    for short, kind in [(True, "lean_top_levels"), (False, "radix_pass")]:
        if short:  # free memory between the two workspaces
            kdb.kdb_debug_inject_fault(kdb.FAULT_LOW_MEMORY, (256 << 20) + (lean_bytes + fast_bytes) // 2)
        d = torch.from_numpy(pts.copy()).cuda()
        kdb.kdb_profile_start()
        kdb.kdb_build(d, 3, kdb.ROUND_ROBIN)
        kinds = {p["name"] for p in kdb.kdb_profile_stop()}
        assert kind in kinds and (("lean_top_levels" in kinds) == short)
        assert d.cpu().numpy().view(np.uint32).tobytes() == want.view(np.uint32).tobytes()
    assert kdb.kdb_debug_inject_fault(kdb.FAULT_NONE, 0) == kdb.FAULT_NONE  # the hook was used up
