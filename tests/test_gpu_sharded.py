"""The sharded single-tree build's device steps on the GPU, through the C ABI:
kdb_build_subtree against the oracle's subtree build, and the whole protocol
with four shards emulated as threads of one process on one GPU (the
collectives done on the host between the threads; no kernel waits on
another), the assembled tree equal to the oracle's build."""
import threading

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2211_00120_gb300 import kdb, sharded, synth

pytestmark = pytest.mark.gpu

RR, WIDEST, TIGHT = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT, kdb.WIDEST_TIGHT


class ThreadComm:
    """The collectives of `world` threads of one process (test infrastructure)."""

    def __init__(self, rank, world, shared):
        self.rank, self.world, self.s = rank, world, shared

    def _exchange(self, value):
        self.s["slots"][self.rank] = value
        self.s["barrier"].wait()
        vals = list(self.s["slots"])
        self.s["barrier"].wait()
        return vals

    def all_reduce(self, t, op):
        vals = self._exchange(t.clone())
        r = vals[0].clone()
        for v in vals[1:]:
            r = r + v if op == "sum" else (torch.minimum(r, v) if op == "min" else torch.maximum(r, v))
        t.copy_(r)

    def all_to_all(self, send, send_counts, recv_counts):
        vals = self._exchange((send, list(send_counts)))
        parts = []
        for src, counts in vals:
            off = sum(counts[:self.rank])
            parts.append(src[off:off + counts[self.rank]])
        return torch.cat(parts)


def run_threads(pts, k, mode, world):
    dev = torch.device("cuda", torch.cuda.current_device())
    bounds = np.linspace(0, len(pts), world + 1).astype(int)
    bounds[1:-1] += np.array([37, -91, 13, 7, -5, 3, 11][:world - 1])  # uneven shards
    shared = {"slots": [None] * world, "barrier": threading.Barrier(world)}
    results, errors = [None] * world, []

    def body(r):
        try:
            torch.cuda.set_device(dev)
            shard = torch.from_numpy(np.ascontiguousarray(pts[bounds[r]:bounds[r + 1]])).to(dev)
            res = sharded.build_sharded(shard, k, mode, ThreadComm(r, world, shared), sharded.CudaSteps(dev))
            res.records = res.records.cpu().numpy()
            results[r] = res
        except BaseException as e:  # noqa: BLE001 - reported below
            errors.append(e)
            shared["barrier"].abort()

    threads = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return sharded.assemble(results, pts.shape[1])


@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
def test_sharded_build_on_gpu_equals_oracle(mode):
    pts = synth.aniso_float4(400_003, seed=11) if mode == WIDEST else synth.mixed(400_003, 3, seed=11)
    out, orig = run_threads(pts, 3, mode, 4)
    want, worig = oracle.build(pts, 3, mode)
    assert np.array_equal(orig, worig)
    assert np.array_equal(out.view(np.uint32), want.view(np.uint32))


def test_sharded_build_on_gpu_int32_and_two_shards():
    pts = synth.int32_uniform(100_000, 3, seed=5)
    pts[::5, 0] = -7
    out, orig = run_threads(pts, 3, TIGHT, 2)
    assert np.array_equal(orig, oracle.build(pts, 3, TIGHT)[1])
    pts2 = synth.uniform(70_001, 2, seed=6)
    out, orig = run_threads(pts2, 2, RR, 8)
    assert np.array_equal(orig, oracle.build(pts2, 2, RR)[1])


@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
def test_build_subtree_equals_oracle(mode):
    pts = synth.aniso_float4(120_001, seed=3) if mode == WIDEST else synth.mixed(120_001, 3, seed=3)
    for first_dim in range(3):
        dom = np.array([1.0, 0.0, 0.5, 90.0, 1.0, 9.0], np.float32) if mode == WIDEST else None
        want, worig = oracle.build_sub(pts, 3, mode, first_dim, dom)
        d = torch.from_numpy(pts).cuda()
        o = torch.empty(len(pts), dtype=torch.int32, device="cuda")
        kdb.kdb_build_subtree(d, 3, mode, first_dim, dom, o)
        assert np.array_equal(o.cpu().numpy(), worig), (mode, first_dim)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_dist_steps_reject_bad_arguments():
    pts = torch.zeros((10, 3), device="cuda")
    tags = torch.zeros(10, dtype=torch.int32, device="cuda")
    hist = torch.zeros((128, 256), dtype=torch.int32, device="cuda")
    dims = torch.zeros(128, dtype=torch.uint8, device="cuda")
    pre = torch.zeros(128, dtype=torch.int64, device="cuda")
    with pytest.raises(kdb.KdbError):  # more than 64 nodes
        kdb.kdb_dist_histogram(pts, 3, RR, tags, 7, dims, pre, 0, 0, hist)
    with pytest.raises(kdb.KdbError):  # prefix bits not a multiple of 8
        kdb.kdb_dist_histogram(pts, 3, RR, tags, 0, dims, pre, 4, 0, hist)
    with pytest.raises(kdb.KdbError):  # a split dimension >= k: device check
        kdb.kdb_dist_histogram(pts, 3, RR, tags, 0, torch.full((1,), 5, dtype=torch.uint8, device="cuda"),
                               pre, 0, 0, hist)
    with pytest.raises(kdb.KdbError):
        kdb.kdb_build_subtree(pts, 3, WIDEST, 0, None)  # the clipped-domain rule needs the root's domain
