"""The paper's level loop on host threads (oracle/paper_cpu.c, a CPU baseline)
against the recursive oracle: the same tree, for every split rule, float32
and int32 coordinates, one thread and many."""
import numpy as np
import pytest

from oracle import oracle, paper_cpu
from paper_2211_00120_gb300 import synth

RR, WIDEST, TIGHT = oracle.ROUND_ROBIN, oracle.WIDEST, oracle.WIDEST_TIGHT


@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("n", [1, 2, 3, 10, 1000, 4097, 70001])
def test_float_equals_oracle(n, threads, mode):
    pts = synth.mixed(n, 3, seed=n) if n > 3 else synth.uniform(n, 3, seed=n)
    assert list(paper_cpu.build(pts, 3, mode, threads)) == list(oracle.build(pts, 3, mode)[1])


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_int32_and_ties_equal_oracle(mode):
    rng = np.random.default_rng(4)
    for k in (1, 2, 3):
        pts = rng.integers(-3, 3, size=(20000, k)).astype(np.int32)
        assert list(paper_cpu.build(pts, k, mode, 8)) == list(oracle.build(pts, k, mode)[1])
        full = rng.integers(-2**31, 2**31, size=(20000, k), dtype=np.int64).astype(np.int32)
        assert list(paper_cpu.build(full, k, mode, 4)) == list(oracle.build(full, k, mode)[1])


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_uint32_equals_oracle(mode):
    rng = np.random.default_rng(6)
    for k in (1, 3):
        full = rng.integers(0, 2**32, size=(20000, k), dtype=np.uint64).astype(np.uint32)
        assert list(paper_cpu.build(full, k, mode, 4)) == list(oracle.build(full, k, mode)[1])


def test_aniso_widest_and_payload():
    pts = synth.aniso_float4(50000, seed=2)
    for mode in (WIDEST, TIGHT):
        assert list(paper_cpu.build(pts, 3, mode, 6)) == list(oracle.build(pts, 3, mode)[1])


def test_nan_is_rejected():
    pts = synth.uniform(100, 3, seed=1)
    pts[5, 1] = np.nan
    with pytest.raises(RuntimeError):
        paper_cpu.build(pts, 3, RR, 2)
