"""Tuning of the two sort kernels (kdb_set_tuning, kdb_autotune, the tuning
table): every compiled tile-shape pair and digit width must give the oracle's
output bit for bit, since a shape only changes how a pass is cut into tiles
and a width how many passes the level-0 sort takes, not what they compute."""
import functools
import itertools

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth
from tests.test_gpu_parity import gpu_build, tie_grid

pytestmark = pytest.mark.gpu

NPART = len(kdb.kdb_tuning_shapes(kdb.TUNE_PARTITION))
NRAD = len(kdb.kdb_tuning_shapes(kdb.TUNE_RADIX))
WIDTHS = kdb.kdb_digit_widths()
PAIRS = list(itertools.product(range(NPART), range(NRAD), WIDTHS))
# every shape of each kernel and every digit width at least once
COVER = sorted({(p, p % NRAD, WIDTHS[p % len(WIDTHS)]) for p in range(NPART)} |
               {(r % NPART, r, WIDTHS[(r + 1) % len(WIDTHS)]) for r in range(NRAD)})


@pytest.fixture(autouse=True)
def default_tuning_after():
    yield
    kdb.kdb_clear_tuning_table()
    kdb.kdb_set_tuning(0, 0)


CASES = {
    # several tiles of every shape and a ragged tail, two to five global levels
    "uniform3": lambda: synth.uniform(300001, 3, seed=17),
    "mixed2": lambda: synth.mixed(65537, 2, seed=5),
    "ties3": lambda: tie_grid(120011, 3, 7, seed=3),
    "int1": lambda: synth.int32_uniform(200003, 1, seed=8),
}
MODES = [oracle.ROUND_ROBIN, oracle.WIDEST, oracle.WIDEST_TIGHT]


@functools.lru_cache(maxsize=None)
def case(name):
    return CASES[name]()


@functools.lru_cache(maxsize=None)
def want(name, k, mode):
    return oracle.build(case(name), k, mode)


def check(name, k, mode):
    pts = case(name)
    wpts, worig = want(name, k, mode)
    got, gorig = gpu_build(pts, k, mode)
    if not np.array_equal(gorig, worig):
        bad = int(np.flatnonzero(gorig != worig)[0])
        raise AssertionError(f"{name} mode={mode} tuning={kdb.kdb_get_tuning()}: node {bad} holds "
                             f"{gorig[bad]}, oracle {worig[bad]}")
    assert got.view(np.uint32).tobytes() == wpts.view(np.uint32).tobytes()


@pytest.mark.parametrize("pair", PAIRS)
def test_every_shape_pair_matches_the_oracle(pair):
    kdb.kdb_set_tuning(*pair)
    check("uniform3", 3, oracle.ROUND_ROBIN)


@pytest.mark.parametrize("pair", COVER)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", ["uniform3", "mixed2", "ties3"])
def test_every_shape_in_every_mode(name, mode, pair):
    k = case(name).shape[1]
    kdb.kdb_set_tuning(*pair)
    check(name, k, mode)


@pytest.mark.parametrize("pair", COVER)
def test_every_shape_int32(pair):
    kdb.kdb_set_tuning(*pair)
    check("int1", 1, oracle.ROUND_ROBIN)


@pytest.mark.parametrize("pair", [p for p in COVER if p != (0, 0, 8)])
def test_batched_sets_under_other_shapes(pair):
    sizes = [9000, 1, 40000, 8191, 8192, 130001, 2, 17000]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = synth.uniform(int(offs[-1]), 3, seed=23)
    kdb.kdb_set_tuning(*pair)
    d = torch.from_numpy(pts.copy()).cuda()
    kdb.kdb_build_batched(d, offs, 3, kdb.ROUND_ROBIN)
    got = d.cpu().numpy()
    for a, b in zip(offs[:-1], offs[1:]):
        w, _ = oracle.build(pts[a:b], 3, oracle.ROUND_ROBIN)
        assert got[a:b].view(np.uint32).tobytes() == w.view(np.uint32).tobytes()


def test_autotune_keeps_the_fastest_choice_and_leaves_points_alone():
    pts = synth.uniform(2_000_000, 3, seed=31)
    d = torch.from_numpy(pts).cuda()
    r = kdb.kdb_autotune(d, 3, kdb.ROUND_ROBIN, reps=3)
    assert set(r["ms"]) == set(PAIRS)
    assert all(v > 0 for v in r["ms"].values())
    assert r["best"] in PAIRS and r["best_ms"] == min(r["ms"].values())
    assert kdb.kdb_get_tuning() == r["best"]
    # kept in the table for builds of this kind
    assert kdb.kdb_lookup_tuning(len(pts), 3, 12, kdb.ROUND_ROBIN) == (r["best"], True)
    assert torch.equal(d.cpu(), torch.from_numpy(pts))  # read only
    # a build under the kept setting is still the oracle's tree
    got, _ = gpu_build(pts, 3, kdb.ROUND_ROBIN)
    w, _ = oracle.build(pts, 3, oracle.ROUND_ROBIN)
    assert got.view(np.uint32).tobytes() == w.view(np.uint32).tobytes()


def test_autotune_times_only_the_current_choice_where_nothing_is_tuned():
    kdb.kdb_set_tuning(*PAIRS[-1])
    # k = 4 builds without the per-dimension lists; 5000 points need no global level
    for pts, k in [(synth.uniform(300000, 4, seed=2), 4), (synth.uniform(5000, 3, seed=2), 3)]:
        r = kdb.kdb_autotune(torch.from_numpy(pts).cuda(), k, kdb.ROUND_ROBIN, reps=1)
        assert list(r["ms"]) == [PAIRS[-1]] and r["best"] == PAIRS[-1]
        assert not kdb.kdb_lookup_tuning(len(pts), k, 4 * k)[1]  # nothing kept


def test_autotune_refuses_bad_arguments():
    d = torch.from_numpy(synth.uniform(1000, 3, seed=1)).cuda()
    for reps in (0, 65):
        with pytest.raises(kdb.KdbError) as e:
            kdb.kdb_autotune(d, 3, kdb.ROUND_ROBIN, reps=reps)
        assert e.value.code == kdb.ERR_INVALID_ARGUMENT
    with pytest.raises(kdb.KdbError):
        kdb.kdb_autotune(d[:1], 3, kdb.ROUND_ROBIN)
    assert kdb.kdb_get_tuning() == (0, 0, 8)


def test_table_entry_drives_builds_of_its_kind():
    """A build takes its kind's table entry: an entry for one size bucket and
    the process-wide setting elsewhere, both the oracle's tree."""
    pts = case("uniform3")
    wpts, _ = want("uniform3", 3, oracle.ROUND_ROBIN)
    d = torch.from_numpy(pts).cuda()
    r = kdb.kdb_autotune(d, 3, kdb.ROUND_ROBIN, reps=1)
    assert kdb.kdb_lookup_tuning(len(pts), 3, 12)[1]
    kdb.kdb_set_tuning(0, 0, 8 if r["best"][2] == 6 else 6)  # the process-wide setting differs
    got, _ = gpu_build(pts, 3, kdb.ROUND_ROBIN)
    assert got.view(np.uint32).tobytes() == wpts.view(np.uint32).tobytes()
    small = pts[:100_000]
    assert not kdb.kdb_lookup_tuning(len(small), 3, 12)[1]
    got, _ = gpu_build(small, 3, kdb.ROUND_ROBIN)
    assert got.view(np.uint32).tobytes() == oracle.build(small, 3, oracle.ROUND_ROBIN)[0].view(np.uint32).tobytes()


def test_table_from_a_file_drives_builds(tmp_path):
    """A 6-bit entry loaded from a file for one kind, 8 bits for the rest:
    builds of both kinds equal the oracle's."""
    part = kdb.kdb_tuning_shapes(kdb.TUNE_PARTITION)
    rad = kdb.kdb_tuning_shapes(kdb.TUNE_RADIX)
    pts = case("ties3")
    entry = {"log2n": int(len(pts)).bit_length(), "k": 3, "stride": 12, "mode": kdb.WIDEST_TIGHT,
             "partition": list(part[1]), "radix": list(rad[1]), "digit_bits": 6}
    f = tmp_path / "t.json"
    import json
    f.write_text(json.dumps({"partition": list(part[0]), "radix": list(rad[0]), "table": [entry]}))
    kdb.kdb_load_tuning(str(f))
    assert kdb.kdb_lookup_tuning(len(pts), 3, 12, kdb.WIDEST_TIGHT) == ((1, 1, 6), True)
    check("ties3", 3, oracle.WIDEST_TIGHT)
    check("ties3", 3, oracle.ROUND_ROBIN)
