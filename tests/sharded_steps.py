"""Host stand-ins for the device steps of the sharded single-tree build
(test infrastructure): the same interface as ``sharded.CudaSteps``, on numpy
arrays, with the oracle's subtree build as the local build.  Lets the
protocol (radix select, domains, exchange) run as gloo processes on the CPU.

Keys follow their definition in the paper's terms: the order-preserving
coordinate key (Sec. 7.1's radix key; -0.0 below +0.0) shifted left by 32,
OR'ed with the point's original index, so the order of keys is the strict
order of Sec. 3.1 with the tie rule."""
import numpy as np
import torch

from oracle import oracle

INT32, UINT32 = 0x100, 0x200


def coord_keys(col: np.ndarray, mode: int) -> np.ndarray:
    bits = np.ascontiguousarray(col).view(np.uint32).astype(np.uint64)
    if mode & UINT32:
        return bits
    if mode & INT32:
        return bits ^ np.uint64(0x80000000)
    neg = (bits & np.uint64(0x80000000)) != 0
    return np.where(neg, bits ^ np.uint64(0xFFFFFFFF), bits ^ np.uint64(0x80000000))


class NumpySteps:
    def count(self, points) -> int:
        return points.shape[0]

    def with_coord_type(self, points, mode: int) -> int:
        if mode & (INT32 | UINT32):
            return mode
        return mode | {np.dtype(np.int32): INT32, np.dtype(np.uint32): UINT32}.get(points.dtype, 0)

    def row_words(self, points) -> int:
        return points.shape[1]

    def tags(self, n: int):
        return np.zeros(n, dtype=np.int32)

    def _key64(self, points, d, base, sel):
        keys = coord_keys(points[sel, d], self.mode)
        return (keys << np.uint64(32)) | (np.uint64(base) + np.flatnonzero(sel).astype(np.uint64))

    def box(self, points, k, mode, tags, level):
        self.mode = mode
        nodes, first = 1 << level, (1 << level) - 1
        box = np.zeros((nodes, 2 * k), dtype=np.int64)
        box[:, :k] = 0xFFFFFFFF
        for u in range(nodes):
            sel = tags == first + u
            if sel.any():
                for d in range(k):
                    keys = coord_keys(points[sel, d], mode).astype(np.int64)
                    box[u, d], box[u, k + d] = keys.min(), keys.max()
        return torch.from_numpy(box)

    def histogram(self, points, k, mode, tags, level, dims, prefix, bits, base):
        self.mode = mode
        nodes, first = 1 << level, (1 << level) - 1
        hist = np.zeros((nodes, 256), dtype=np.int64)
        for u in range(nodes):
            sel = tags == first + u
            key = self._key64(points, dims[u], base, sel)
            if bits:
                key = key[(key >> np.uint64(64 - bits)) == np.uint64(prefix[u])]
            hist[u] = np.bincount(((key >> np.uint64(56 - bits)) & np.uint64(255)).astype(np.int64),
                                  minlength=256)
        return torch.from_numpy(hist)

    def assign(self, points, k, mode, tags, level, dims, pivot, base):
        self.mode = mode
        nodes, first = 1 << level, (1 << level) - 1
        pinned = np.full(nodes, -1, dtype=np.int64)
        new = tags.copy()
        for u in range(nodes):
            sel = tags == first + u
            where = np.flatnonzero(sel)
            key = self._key64(points, dims[u], base, sel)
            piv = np.uint64(pivot[u])
            t = first + u
            new[where[key < piv]] = 2 * t + 1
            new[where[key > piv]] = 2 * t + 2
            hit = where[key == piv]
            if len(hit):
                new[hit] = -1
                pinned[u] = int(hit[0])
        tags[:] = new
        return pinned

    def record_words(self, points, i):
        return points[i].view(np.int32).astype(np.int64)

    def partition(self, points, tags, first, ndest, base):
        dest = tags.astype(np.int64) - first
        sel = (dest >= 0) & (dest < ndest)
        ids = np.flatnonzero(sel)
        order = ids[np.argsort(dest[sel], kind="stable")]
        out = np.ascontiguousarray(points[order])
        idx = torch.from_numpy((order + base).astype(np.int32))
        counts = [int(c) for c in np.bincount(dest[sel], minlength=ndest)]
        return out, idx, counts

    def as_bytes(self, records):
        return torch.from_numpy(np.ascontiguousarray(records).view(np.uint8).reshape(-1).copy())

    def from_bytes(self, raw, like, rows):
        return raw.numpy().view(like.dtype).reshape(rows, like.shape[1]).copy()

    def int_tensor(self, values):
        return torch.from_numpy(np.array(values, dtype=np.int64))

    def build_subtree(self, points, k, mode, first_dim, domain):
        out, orig = oracle.build_sub(points, k, mode, first_dim, domain)
        return out, orig

    def to_host(self, x):
        return x.numpy() if isinstance(x, torch.Tensor) else np.asarray(x)
