"""Step-by-step CPU emulator of the paper's level loop (test infrastructure only).

This follows the algorithm of Sec. 3 in the paper's own order and notation:
every point carries a tag (its level-l ancestor, Sec. 2.2), initialised to 0;
each iteration l sorts the whole array with the ``less()`` order of Sec. 3.1
(tag first, then the coordinate in the split dimension) and then runs the tag
update of Sec. 3.2, which uses the O(1) sub-tree size ``ss`` (Sec. 4.1) and
segment begin ``sb`` (Sec. 4.2).  After L-1 iterations a final sort by tag puts
every point at its node.  The split-widest extension (Sec. 6) keeps a split
dimension per subtree; it is stored in a dict keyed by node id instead of the
low tag bits, which changes nothing about the order.

Readings where the paper is silent or garbled:
  * equal keys: ``less()`` alone is not a strict order; ties go to the lower
    original index, and -0.0 sorts before +0.0;
  * the listings in Sec. 4 write ``1<<(L-l-1) - 1``, which C parses as a shift
    by L-l-2; the intended value (and the one used here) is
    ``(1<<(L-l-1)) - 1``.  ``ss_literal``/``sb_literal`` keep the C reading so
    a test can show it disagrees with the subtree sizes;
  * the loop bound ``for l = 0 .. log2(N)``: L-1 = floor(log2 N) sort+update
    iterations, then the final sort, as in the Sec. 5 walkthrough;
  * clipping a subtree's box by a plane (Sec. 6) means ``hi = min(hi, x)`` on
    the left side and ``lo = max(lo, x)`` on the right;
  * widest dimension: argmax of hi-lo in float32 with a strict '>' from d=0.

A third split rule, which the paper does not have, is emulated as well:
``WIDEST_TIGHT`` takes the widest side of each subtree's tight bounding box,
the min/max over the points that carry the subtree's tag after the update (a
segmented reduction over each tag's points).

It is the emulator of the paper's algorithm, not the oracle proper (that is the
recursive builder in ``kd_oracle.c``); tests check the two against each other.
"""
from __future__ import annotations

import math

import numpy as np

ROUND_ROBIN = 0
WIDEST = 1
WIDEST_TIGHT = 2


def num_levels(n: int) -> int:
    """L = numLevels(N) = 32 - clz(N) (Sec. 2, corrected in Revision 3)."""
    return n.bit_length()


def level(i: int) -> int:
    """level(i) = 31 - clz(i+1) (Sec. 2)."""
    return (i + 1).bit_length() - 1


def F(l: int) -> int:
    """Nodes in a full tree of l levels: 2^l - 1 (Sec. 2)."""
    return (1 << l) - 1


def ss(s: int, n: int) -> int:
    """Sub-tree size in O(1) (Sec. 4.1): full inner levels plus the part of
    the lowest level that lies below s."""
    L = num_levels(n)
    l = level(s)
    h = L - l - 1
    fllc = ~((~s) << h)  # append h one-bits: first lowest-level child
    inner = (1 << h) - 1
    lowest = min(max(0, n - fllc), 1 << h)
    return inner + lowest


def sb(s: int, l: int, n: int) -> int:
    """Segment begin of subtree s after the level-l sort, O(1) (Sec. 4.2)."""
    L = num_levels(n)
    nls = s - ((1 << l) - 1)  # left siblings of s on level l
    h = L - l - 1
    return ((1 << l) - 1) + nls * ((1 << h) - 1) + min(nls * (1 << h), n - ((1 << (L - 1)) - 1))


def _shift(a: int, b: int) -> int:
    return a << b if b >= 0 else a >> (-b)


def ss_literal(s: int, n: int) -> int:
    """Sec. 4.1's snippet read with C precedence: ``1<<(L-l-1) - 1`` shifts
    by L-l-2.  Kept only to show that this reading is wrong."""
    L = num_levels(n)
    l = level(s)
    h = L - l - 1
    fllc = ~((~s) << h)
    return _shift(1, h - 1) + min(max(0, n - fllc), 1 << h)


def _fkey(v: float):
    """Sort key for a float32 value: numeric order with -0.0 before +0.0."""
    return (v, 0 if math.copysign(1.0, v) < 0 else 1)


def _widest(lo, hi) -> int:
    if all(isinstance(v, int) for v in list(lo) + list(hi)):
        ext = [h - lo_ for lo_, h in zip(lo, hi)]  # integer coordinates: exact
    else:
        ext = [np.float32(h) - np.float32(lo_) for lo_, h in zip(lo, hi)]
    best = 0
    for d in range(1, len(ext)):
        if ext[d] > ext[best]:
            best = d
    return best


def emulate(points: np.ndarray, k: int, mode: int = ROUND_ROBIN, trace=None):
    """Runs the level loop on ``points`` (rows = records, first k columns =
    float32 coordinates).  Returns the original index of the point at each
    node.  ``trace(step, l, tags, order)`` is called after every sort and
    every update (step in {"sort", "update", "final"})."""
    # integer coordinates: int32 (Sec. 5 uses int2) or uint32
    ints = np.asarray(points).dtype in (np.int32, np.uint32)
    P = np.asarray(points) if ints else np.asarray(points, dtype=np.float32)
    n = P.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    conv = int if ints else float
    coords = [[conv(P[i, d]) for d in range(k)] for i in range(n)]
    arr = [[0, i] for i in range(n)]  # [tag, original index]
    L = num_levels(n)
    dims = {}
    if mode in (WIDEST, WIDEST_TIGHT):
        lo = [min((coords[i][d] for i in range(n)), key=_fkey) for d in range(k)]
        hi = [max((coords[i][d] for i in range(n)), key=_fkey) for d in range(k)]
        scene = (lo, hi)
        dims[0] = _widest(lo, hi)

    def dim_of(tag: int, l: int) -> int:
        return l % k if mode == ROUND_ROBIN else dims[tag]

    for l in range(L - 1):
        # parallel sort {tags, points} with less(): (tag, coordinate, index)
        arr.sort(key=lambda e: (e[0], _fkey(coords[e[1]][dim_of(e[0], l)]), e[1]))
        if trace:
            trace("sort", l, [e[0] for e in arr], [e[1] for e in arr])
        # updateTags (Sec. 3.2)
        new_subtrees = set()
        for i in range(n):
            if i < F(l):
                continue
            s = arr[i][0]
            pivot = sb(s, l, n) + ss(2 * s + 1, n)
            if i < pivot:
                arr[i][0] = 2 * s + 1
            elif i > pivot:
                arr[i][0] = 2 * s + 2
            else:
                continue
            new_subtrees.add((arr[i][0], s, pivot))
        if mode == WIDEST:
            # split dimension of each new subtree: scene box clipped by the
            # plane of s, then by every ancestor of s on the way to the root
            for child, s, pivot in sorted(new_subtrees):
                blo, bhi = list(scene[0]), list(scene[1])

                def clip(node_coords, d, left):
                    x = node_coords[d]
                    if left:
                        bhi[d] = min(bhi[d], x, key=_fkey)
                    else:
                        blo[d] = max(blo[d], x, key=_fkey)

                clip(coords[arr[pivot][1]], dims[s], child == 2 * s + 1)
                t = s
                while t > 0:
                    p = (t - 1) // 2
                    # p was fixed in an earlier iteration: after this
                    # iteration's sort it sits at array slot p
                    clip(coords[arr[p][1]], dims[p], t == 2 * p + 1)
                    t = p
                dims[child] = _widest(blo, bhi)
        if mode == WIDEST_TIGHT:
            # each new subtree's box: min / max over the points now tagged with it
            members = {}
            for tag, o in arr:
                members.setdefault(tag, []).append(o)
            for child, _, _ in new_subtrees:
                ms = members[child]
                blo = [min((coords[o][d] for o in ms), key=_fkey) for d in range(k)]
                bhi = [max((coords[o][d] for o in ms), key=_fkey) for d in range(k)]
                dims[child] = _widest(blo, bhi)
        if trace:
            trace("update", l, [e[0] for e in arr], [e[1] for e in arr])
    arr.sort(key=lambda e: e[0])
    if trace:
        trace("final", L - 1, [e[0] for e in arr], [e[1] for e in arr])
    return np.array([e[1] for e in arr], dtype=np.int64)
