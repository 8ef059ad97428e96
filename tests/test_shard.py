"""Sharding of batched sets over ranks (host logic), and the multi-rank
batched path run as world-size-2 gloo processes on the CPU with the oracle
standing in for each rank's GPU build: the assembled result must equal the
oracle over all sets, and every rank must compute the same assignment."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_00120_gb300 import shard, synth


def test_lpt_covers_every_set_once_and_balances():
    sizes = [int(s) for s in synth.lognormal_sizes(4096, 100, 1e6, seed=3)]
    for world in (1, 2, 3, 4, 8):
        shards = shard.lpt_shards(sizes, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(sizes)))
        loads = [shard.shard_cost(sizes, s) for s in shards]
        # LPT bound: no rank exceeds the average by more than the largest set
        assert max(loads) <= sum(loads) / world + max(shard.build_cost(n) for n in sizes)


def test_lpt_is_deterministic_and_handles_empty_sets():
    sizes = [0, 5, 5, 0, 1, 7, 7, 7, 3]
    a = shard.lpt_shards(sizes, 3)
    assert a == shard.lpt_shards(list(sizes), 3)
    assert sorted(i for s in a for i in s) == list(range(len(sizes)))
    with pytest.raises(ValueError):
        shard.lpt_shards(sizes, 0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, sizes, pts, out_dir):
    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    mine = shard.lpt_shards(sizes, world)[rank]
    built = {}
    for b in mine:  # this rank's share; on a GPU this is one kdb_build_batched call
        lo, hi = offs[b], offs[b + 1]
        if hi > lo:
            built[b] = oracle.build(pts[lo:hi], 3, oracle.ROUND_ROBIN)[0]
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, built))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.array(gathered, dtype=object),
                allow_pickle=True)
    dist.destroy_process_group()


def test_two_ranks_build_their_shares_and_match_the_oracle(tmp_path):
    from oracle import oracle
    oracle.compile_oracle()
    sizes = [int(s) for s in synth.lognormal_sizes(24, 10, 400, seed=5)] + [0, 1]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = synth.uniform(int(offs[-1]), 3, seed=6)
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), sizes, pts, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    gathered = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    seen = []
    for mine, built in gathered:
        seen += list(mine)
        for b, out in built.items():
            lo, hi = offs[b], offs[b + 1]
            want = oracle.build(pts[lo:hi], 3, oracle.ROUND_ROBIN)[0]
            assert np.array_equal(out.view(np.uint32), want.view(np.uint32))
    assert sorted(seen) == list(range(len(sizes)))
    # each rank's share is the deterministic assignment
    assert [list(m) for m, _ in gathered] == shard.lpt_shards(sizes, world)


def test_uniform_rows_equal_slices_of_the_whole_draw():
    whole = synth.uniform(5000, 3, seed=3)
    for start, n in [(0, 10), (17, 100), (4990, 10), (1234, 0)]:
        assert np.array_equal(synth.uniform_rows(start, n, 3, seed=3), whole[start:start + n])
