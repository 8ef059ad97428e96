"""Plans (kdb_plan_*): a build prepared once and enqueued many times, and
captured into a CUDA graph that is replayed on new point data.  Every output
must equal the oracle's (exact)."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, synth

pytestmark = pytest.mark.gpu

RR, WIDEST = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT


def oracle_sets(pts, offs, k, mode):
    out = np.empty_like(pts)
    for b in range(len(offs) - 1):
        lo, hi = offs[b], offs[b + 1]
        if hi > lo:
            out[lo:hi] = oracle.build(pts[lo:hi], k, mode)[0]
    return out


@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_plan_enqueue_repeats_equal_oracle(mode):
    n = 150001
    plan = kdb.Plan(n, 3, 12, mode)
    assert plan.workspace_bytes > 0
    for seed in (1, 2, 3):
        pts = synth.mixed(n, 3, seed=seed)
        d = torch.from_numpy(pts).cuda()
        plan.enqueue(d)
        plan.status()
        want = oracle.build(pts, 3, mode)[0]
        assert np.array_equal(d.cpu().numpy().view(np.uint32), want.view(np.uint32))
    plan.close()


@pytest.mark.parametrize("mode", [RR, WIDEST])
def test_plan_captured_in_cuda_graph_and_replayed(mode):
    sizes = [3, 40000, 0, 9000, 1, 70001, 500]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    plan = kdb.Plan(offs.tolist(), 3, 12, mode)
    buf = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    src = torch.empty_like(buf)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            buf.copy_(src)                # the input copy is part of the graph
            plan.enqueue(buf, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for seed in (11, 12):
        pts = synth.uniform(n, 3, seed=seed)
        src.copy_(torch.from_numpy(pts))
        g.replay()
        torch.cuda.synchronize()
        plan.status()
        want = oracle_sets(pts, offs, 3, mode)
        assert np.array_equal(buf.cpu().numpy().view(np.uint32), want.view(np.uint32))
    del g
    plan.close()


def test_plan_reports_nan_through_status():
    n = 20000
    plan = kdb.Plan(n, 3, 12, RR)
    pts = synth.uniform(n, 3, seed=4)
    pts[123, 2] = np.nan
    d = torch.from_numpy(pts).cuda()
    plan.enqueue(d)
    with pytest.raises(kdb.KdbError) as e:
        plan.status()
    assert e.value.code == kdb.ERR_NAN_INPUT
    assert np.array_equal(d.cpu().numpy().view(np.uint32), pts.view(np.uint32))
    plan.close()
