"""Sharded single-tree build: one left-balanced k-d tree over points held by
several processes, one GPU each.

The paper builds the tree on one GPU by whole-array sorts (Sec. 3, 7.2).
Here the array is split into shards, shard r holding the global records
[base_r, base_r + n_r).  For G = 2^g shards:

  1. The top g levels are built across the shards, level by level, as the
     paper's level step (Sec. 3): every node's pivot is the point of rank
     ss(lChild) in the node's order by (coordinate, original index)
     (Observation 1), found by a radix select over the 64-bit key
     (coordinate key << 32 | original index) whose digit histograms are
     summed over the shards (one all-reduce per 8 bits); every point's tag
     then moves to the child on its side (Sec. 3.2).  The split dimension
     is round robin, the widest side of the node's domain (Sec. 6, domains
     carried top-down on the host) or the widest side of the node's tight
     box (boxes reduced over the shards).
  2. One exchange sends every point to the shard that owns its level-g
     subtree (all-to-all), in original-index order.
  3. Every shard builds its subtree alone (kdb_build_subtree): a subtree of a
     left-balanced complete tree is itself one of its size, with the split
     rule continued from its root.

Everything the GPU does goes through the library's C ABI (``kdb.kdb_dist_*``,
``kdb.kdb_build_subtree``); this module holds the host logic: the radix
select's bucket choice, the domains, the exchange plan.  The collectives come
from ``comm`` (``TorchComm`` over ``torch.distributed``: NCCL between GPUs,
gloo for the CPU tests) and the device steps from ``steps`` (``CudaSteps``);
both are parameters so that the same protocol can be driven with other
implementations of the two interfaces.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import kdb

ROUND_ROBIN, WIDEST_EXTENT, WIDEST_TIGHT = kdb.ROUND_ROBIN, kdb.WIDEST_EXTENT, kdb.WIDEST_TIGHT


def full_nodes(l: int) -> int:
    """F(l) = 2^l - 1: nodes above level l (Sec. 2)."""
    return (1 << l) - 1


def subtree_size(s: int, n: int) -> int:
    """ss(s) (Sec. 4.1): nodes of the subtree at s in a tree of n nodes."""
    if s >= n:
        return 0
    L = n.bit_length()
    h = L - ((s + 1).bit_length() - 1) - 1
    w = 1 << h
    fllc = (s << h) + (w - 1)  # the subtree's first slot on the lowest level
    low = 0 if fllc >= n else min(n - fllc, w)
    return (w - 1) + low


def key_to_float(key: int) -> np.float32:
    """Inverse of the order-preserving float key (Sec. 7.1's radix key)."""
    bits = key ^ (0x80000000 if key & 0x80000000 else 0xFFFFFFFF)
    return np.array([bits], dtype=np.uint32).view(np.float32)[0]


def widest(lo, hi, k: int, ints: bool) -> int:
    """Widest side of a box: float32 hi - lo (integers: exact differences),
    strict '>' from d = 0, so the lowest dimension wins ties."""
    best, be = 0, None
    for d in range(k):
        e = int(hi[d]) - int(lo[d]) if ints else np.float32(hi[d]) - np.float32(lo[d])
        if d == 0 or e > be:
            best, be = d, e
    return best


@dataclass
class ShardResult:
    """One shard's part of the tree: the top nodes (the same on every shard)
    and the subtree this shard owns, in its own level order."""
    top_records: np.ndarray      # F(g) records of the top levels, in level order (host)
    top_orig: np.ndarray         # their original indices
    root: int                    # the owned subtree's root node (F(g) + rank)
    records: object              # the subtree's records in its level order (steps' array type)
    orig: np.ndarray             # original index of each of them (host)
    levels: int                  # g, the levels built across the shards
    n: int                       # N, points in the whole tree


def subtree_node_ids(root: int, m: int, g: int, rank: int) -> np.ndarray:
    """Global node of each node of the subtree at level g owned by `rank`,
    given in the subtree's own level order (m nodes): local node q on local
    level lam = level(q) is node F(g + lam) + (rank << lam) + (q - F(lam))."""
    q = np.arange(m, dtype=np.int64)
    lam = np.zeros(m, dtype=np.int64)  # level(q) = bit length of q + 1, minus one
    v = q + 1
    for b in range(5, -1, -1):
        step = 1 << b
        big = v >= np.left_shift(np.int64(1), step)
        lam += np.where(big, step, 0)
        v = np.where(big, np.right_shift(v, step), v)
    one = np.int64(1)
    return (np.left_shift(one, g + lam) - 1) + np.left_shift(np.int64(rank), lam) + (q - (np.left_shift(one, lam) - 1))


class TorchComm:
    """The collectives over ``torch.distributed`` (NCCL between GPUs, gloo on
    the CPU); tensors live on ``device``."""

    def __init__(self, device, group=None):
        import torch.distributed as dist

        self.dist, self.group, self.device = dist, group, device
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def all_reduce(self, t, op: str):
        ops = {"sum": self.dist.ReduceOp.SUM, "min": self.dist.ReduceOp.MIN, "max": self.dist.ReduceOp.MAX}
        self.dist.all_reduce(t, op=ops[op], group=self.group)

    def all_to_all(self, send, send_counts, recv_counts):
        import torch

        out = torch.empty(sum(recv_counts), dtype=send.dtype, device=send.device)
        self.dist.all_to_all_single(out, send, list(recv_counts), list(send_counts), group=self.group)
        return out


class CudaSteps:
    """The device steps on this process's GPU, through the library's C ABI.
    Points are a 2-D CUDA tensor of 4-byte items (one row per record)."""

    def __init__(self, device):
        import torch

        self.torch, self.device = torch, torch.device(device)

    def count(self, points) -> int:
        return int(points.shape[0])

    def with_coord_type(self, points, mode: int) -> int:
        return kdb._mode(points, mode)

    def row_words(self, points) -> int:
        return int(points.shape[1])

    def tags(self, n: int):
        return self.torch.zeros(n, dtype=self.torch.int32, device=self.device)

    def _dev(self, a, dtype):
        return self.torch.as_tensor(np.asarray(a), device=self.device).to(dtype)

    def box(self, points, k, mode, tags, level):
        t = self.torch
        box = t.empty((1 << level, 2 * k), dtype=t.int32, device=self.device)
        kdb.kdb_dist_box(points, k, mode, tags, level, box)
        return box.view(t.int32).to(t.int64) & 0xFFFFFFFF

    def histogram(self, points, k, mode, tags, level, dims, prefix, bits, base):
        t = self.torch
        hist = t.empty((1 << level, 256), dtype=t.int32, device=self.device)
        kdb.kdb_dist_histogram(points, k, mode, tags, level, self._dev(dims, t.uint8),
                               self._dev(np.array(prefix, np.uint64).view(np.int64), t.int64), bits, base, hist)
        return hist.to(t.int64)

    def assign(self, points, k, mode, tags, level, dims, pivot, base):
        t = self.torch
        pinned = t.full((1 << level,), -1, dtype=t.int64, device=self.device)
        kdb.kdb_dist_assign(points, k, mode, tags, level, self._dev(dims, t.uint8),
                            self._dev(np.array(pivot, np.uint64).view(np.int64), t.int64), base, pinned)
        return pinned.cpu().numpy()

    def record_words(self, points, i: int) -> np.ndarray:
        return points[i].view(self.torch.int32).cpu().numpy().astype(np.int64)

    def partition(self, points, tags, first, ndest, base):
        t = self.torch
        out = t.empty_like(points)
        idx = t.empty(points.shape[0], dtype=t.int32, device=self.device)
        counts = kdb.kdb_dist_partition(points, tags, first, ndest, base, out, idx)
        return out, idx, counts

    def as_bytes(self, records):
        return records.contiguous().view(self.torch.uint8).reshape(-1)

    def from_bytes(self, raw, like, rows: int):
        return raw.view(like.dtype).reshape(rows, like.shape[1])

    def int_tensor(self, values):
        return self.torch.as_tensor(np.asarray(values, np.int64), device=self.device)

    def build_subtree(self, points, k, mode, first_dim, domain):
        t = self.torch
        orig = t.empty(points.shape[0], dtype=t.int32, device=self.device)
        kdb.kdb_build_subtree(points, k, mode, first_dim, domain, orig)
        return points, orig.cpu().numpy()

    def to_host(self, x):
        return x.cpu().numpy()


def build_sharded(points, k: int, mode: int, comm, steps) -> ShardResult:
    """Builds the tree over all shards' points; every process calls this with
    its own shard and receives its part (``ShardResult``)."""
    G, r = comm.world, comm.rank
    if G & (G - 1) or G > 64:
        raise ValueError("the number of shards must be a power of two, at most 64")
    mode = steps.with_coord_type(points, mode)  # int32 / uint32 records carry their type
    split = mode & 0xFF
    ints = bool(mode & (kdb.COORDS_INT32 | kdb.COORDS_UINT32))
    g = G.bit_length() - 1
    n_r = steps.count(points)
    sizes = steps.int_tensor([n_r if j == r else 0 for j in range(G)])
    comm.all_reduce(sizes, "sum")
    sizes = [int(v) for v in steps.to_host(sizes)]
    N, base = sum(sizes), sum(sizes[:r])
    if g > 0 and g > N.bit_length() - 2:
        raise ValueError(f"{N} points are too few for {G} shards: the top {g} levels must be full")
    words = steps.row_words(points)
    tags = steps.tags(n_r)
    top_records = np.zeros((full_nodes(g), words), dtype=np.int64)
    top_orig = np.zeros(full_nodes(g), dtype=np.int64)
    domains = {}
    if split == WIDEST_EXTENT:
        box = steps.box(points, k, mode, tags, 0)
        lo, hi = box[:, :k].clone(), box[:, k:].clone()
        comm.all_reduce(lo, "min")
        comm.all_reduce(hi, "max")
        lo, hi = steps.to_host(lo)[0], steps.to_host(hi)[0]
        domains[0] = (np.array([key_to_float(int(v)) for v in lo], np.float32),
                      np.array([key_to_float(int(v)) for v in hi], np.float32))
    for l in range(g):
        nodes, first = 1 << l, full_nodes(l)
        # the split dimension of every node of the level
        if split == ROUND_ROBIN:
            dims = [l % k] * nodes
        elif split == WIDEST_EXTENT:
            dims = [widest(*domains[first + u], k, False) for u in range(nodes)]
        else:
            box = steps.box(points, k, mode, tags, l)
            lo, hi = box[:, :k].clone(), box[:, k:].clone()
            comm.all_reduce(lo, "min")
            comm.all_reduce(hi, "max")
            lo, hi = steps.to_host(lo), steps.to_host(hi)
            if ints:
                dims = [widest(lo[u], hi[u], k, True) for u in range(nodes)]
            else:
                dims = [widest([key_to_float(int(v)) for v in lo[u]], [key_to_float(int(v)) for v in hi[u]], k,
                               False) for u in range(nodes)]
        # the pivot's rank in its node (Observation 1), then a radix select
        remaining = [subtree_size(2 * (first + u) + 1, N) for u in range(nodes)]
        prefix = [0] * nodes
        for rnd in range(8):
            h = steps.histogram(points, k, mode, tags, l, dims, prefix, 8 * rnd, base)
            comm.all_reduce(h, "sum")
            h = steps.to_host(h)
            for u in range(nodes):
                cum = np.cumsum(h[u])
                dgt = int(np.searchsorted(cum, remaining[u], side="right"))
                if dgt > 255:
                    raise RuntimeError("radix select lost its pivot: the shards disagree")
                remaining[u] -= int(cum[dgt - 1]) if dgt else 0
                prefix[u] = (prefix[u] << 8) | dgt
        pinned = steps.assign(points, k, mode, tags, l, dims, prefix, base)
        # the pivots' records, from the shards that hold them
        recs = np.zeros((nodes, words), dtype=np.int64)
        for u in range(nodes):
            if pinned[u] >= 0:
                recs[u] = steps.record_words(points, int(pinned[u]))
        rt = steps.int_tensor(recs)
        comm.all_reduce(rt, "sum")
        top_records[first:first + nodes] = steps.to_host(rt)
        top_orig[first:first + nodes] = [p & 0xFFFFFFFF for p in prefix]
        if split == WIDEST_EXTENT:
            for u in range(nodes):
                lo, hi = domains.pop(first + u)
                plane = key_to_float(prefix[u] >> 32)
                clo, chi = lo.copy(), hi.copy()
                chi[dims[u]] = plane
                domains[2 * (first + u) + 1] = (lo.copy(), chi)
                clo[dims[u]] = plane
                domains[2 * (first + u) + 2] = (clo, hi.copy())
    # the exchange: every point to the shard owning its level-g subtree
    out, idx, counts = steps.partition(points, tags, full_nodes(g), G, base)
    ct = steps.int_tensor([[counts[j] if i == r else 0 for j in range(G)] for i in range(G)])
    comm.all_reduce(ct, "sum")
    ct = steps.to_host(ct)
    recv_counts = [int(ct[i][r]) for i in range(G)]
    sent = sum(counts)
    rows = comm.all_to_all(steps.as_bytes(out[:sent]), [c * words * 4 for c in counts],
                           [c * words * 4 for c in recv_counts])
    ridx = comm.all_to_all(idx[:sent], counts, recv_counts)
    m = sum(recv_counts)
    root = full_nodes(g) + r
    if m != subtree_size(root, N):
        raise RuntimeError(f"shard {r} received {m} points for a subtree of {subtree_size(root, N)}")
    local = steps.from_bytes(rows, points, m)
    dom = None
    if split == WIDEST_EXTENT:
        lo, hi = domains[root]
        dom = np.concatenate([lo, hi])
    local, lorig = steps.build_subtree(local, k, mode, g % k, dom)
    ridx = steps.to_host(ridx).astype(np.int64) & 0xFFFFFFFF
    return ShardResult(top_records=top_records.astype(np.uint32).view(np.int32), top_orig=top_orig, root=root,
                       records=local, orig=ridx[lorig] if m else ridx[:0], levels=g, n=N)


def assemble(results, words: int) -> tuple[np.ndarray, np.ndarray]:
    """The whole tree (records as int32 words, original indices) from every
    shard's ShardResult, in rank order (host arrays): a convenience for
    checks and for callers that want the tree in one place."""
    N = results[0].n
    g = results[0].levels
    out = np.zeros((N, words), dtype=np.int32)
    orig = np.zeros(N, dtype=np.int64)
    F = full_nodes(g)
    out[:F] = results[0].top_records
    orig[:F] = results[0].top_orig
    for rank, res in enumerate(results):
        recs = np.asarray(res.records).reshape(-1, words).view(np.int32)
        ids = subtree_node_ids(res.root, recs.shape[0], g, rank)
        out[ids] = recs
        orig[ids] = res.orig
    return out, orig
