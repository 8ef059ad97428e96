"""The sharded single-tree build as gloo processes on the CPU: 2 and 4 shards
of one point set, the top levels chosen across the shards (radix select of
the pivots, Observation 1), one exchange, every subtree built alone (the
oracle standing in for each shard's local build), and the assembled tree
equal to the oracle's build of the whole set, in all three split rules."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle
from paper_2211_00120_gb300 import sharded, synth
from tests.sharded_steps import NumpySteps

RR, WIDEST, TIGHT = 0, 1, 2


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def shard_bounds(n: int, world: int, seed: int):
    """Uneven shard sizes that add up to n."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, world)
    cuts = np.round(np.cumsum(w) / w.sum() * n).astype(int)
    return np.concatenate([[0], cuts])


def worker(rank, world, port, pts, k, mode, seed, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = shard_bounds(len(pts), world, seed)
        comm = sharded.TorchComm(torch.device("cpu"))
        res = sharded.build_sharded(np.ascontiguousarray(pts[b[rank]:b[rank + 1]]), k, mode, comm, NumpySteps())
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), top_records=res.top_records, top_orig=res.top_orig,
                 root=res.root, records=np.asarray(res.records), orig=res.orig, levels=res.levels, n=res.n)
    finally:
        dist.destroy_process_group()


def run_sharded(tmp_path, pts, k, mode, world, seed=0):
    mp.start_processes(worker, args=(world, free_port(), pts, k, mode, seed, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    results = []
    for r in range(world):
        z = np.load(tmp_path / f"r{r}.npz")
        results.append(sharded.ShardResult(top_records=z["top_records"], top_orig=z["top_orig"],
                                           root=int(z["root"]), records=z["records"], orig=z["orig"],
                                           levels=int(z["levels"]), n=int(z["n"])))
    return sharded.assemble(results, pts.shape[1])


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
def test_sharded_build_equals_oracle(tmp_path, world, mode):
    if mode == WIDEST:
        pts = synth.aniso_float4(30001, seed=7)  # payload column rides along
    else:
        pts = synth.mixed(30001, 3, seed=7)  # clusters and exact duplicates
    out, orig = run_sharded(tmp_path, pts, 3, mode, world, seed=world)
    want, worig = oracle.build(pts, 3, mode)
    assert np.array_equal(orig, worig)
    assert np.array_equal(out.view(np.uint32), want.view(np.uint32))


def test_sharded_build_int32_tight_and_k2(tmp_path):
    pts = synth.int32_uniform(20000, 3, seed=3)
    pts[::7, 1] = 5  # many ties in one dimension
    out, orig = run_sharded(tmp_path, pts, 3, TIGHT, 4, seed=1)  # the type comes from the dtype
    want, worig = oracle.build(pts, 3, TIGHT)
    assert np.array_equal(orig, worig)
    pts2 = synth.uniform(5000, 2, seed=4)
    out, orig = run_sharded(tmp_path, pts2, 2, RR, 4, seed=2)
    assert np.array_equal(orig, oracle.build(pts2, 2, RR)[1])


def test_subtree_node_ids_and_sizes():
    """The owned subtree's nodes map to their places in the whole tree, and
    the shards' subtree sizes add up (against the oracle's counted sizes)."""
    n, g = 1000, 2
    ids = np.concatenate([sharded.subtree_node_ids(3 + r, oracle.subtree_size(3 + r, n), g, r) for r in range(4)])
    assert sorted(ids.tolist()) == list(range(3, n))
    for s in range(n):
        assert sharded.subtree_size(s, n) == oracle.subtree_size(s, n)
