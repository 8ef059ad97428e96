"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
printed worked example, brute force over all arrangements, a textbook closed
form, or an invariant.  The plausible mistakes these catch: a wrong pivot rank
(Fig. 1, Sec. 5, brute force), a swapped left/right side (brute force,
planted errors), a wrong split dimension (Sec. 5 uses both dimensions; widest
brute force), a broken tie rule (tie-heavy brute force, signed zero), a wrong
subtree size (recursive definition), a dropped payload (bytewise checks).
"""
import itertools
import math
import random

import numpy as np
import pytest

from oracle import emulator, oracle
from paper_2211_00120_gb300 import synth
from tests.golden_io import fig1, tight_box, walkthrough

RR, WIDEST, TIGHT = oracle.ROUND_ROBIN, oracle.WIDEST, oracle.WIDEST_TIGHT


# ---------------------------------------------------------------- helpers --
def fkey(v):
    if isinstance(v, (int, np.integer)):
        return (int(v), 1)  # int32 coordinates: plain integer order
    v = float(v)
    return (v, 0 if math.copysign(1.0, v) < 0 else 1)


def extent(lo, hi):
    if isinstance(lo, (int, np.integer)):
        return int(hi) - int(lo)  # exact for int32 coordinates
    return np.float32(hi) - np.float32(lo)


def strict_less(pts, a, b, d):
    return (fkey(pts[a, d]), a) < (fkey(pts[b, d]), b)


def level(i):
    return (i + 1).bit_length() - 1


def dims_of_arrangement(pts, order, k, mode):
    """Split dimension of every node of the arrangement ``order`` (node ->
    original index): round robin by level, or widest extent of the scene box
    clipped top-down by the ancestors' planes."""
    n = len(order)
    if mode == RR:
        return [level(i) % k for i in range(n)]
    if mode == TIGHT:
        # widest side of the box of the points in node s's subtree
        dims = []
        for s in range(n):
            sub, frontier = [], [s]
            while frontier:
                t = frontier.pop()
                if t < n:
                    sub.append(order[t])
                    frontier += [2 * t + 1, 2 * t + 2]
            lo = [min((pts[o, d] for o in sub), key=fkey) for d in range(k)]
            hi = [max((pts[o, d] for o in sub), key=fkey) for d in range(k)]
            ext = [extent(lo[d], hi[d]) for d in range(k)]
            best = 0
            for d in range(1, k):
                if ext[d] > ext[best]:
                    best = d
            dims.append(best)
        return dims
    lo = [min((pts[i, d] for i in range(n)), key=fkey) for d in range(k)]
    hi = [max((pts[i, d] for i in range(n)), key=fkey) for d in range(k)]
    dims = [0] * n
    boxes = {0: (list(lo), list(hi))}
    for s in range(n):
        blo, bhi = boxes[s]
        ext = [np.float32(bhi[d]) - np.float32(blo[d]) for d in range(k)]
        best = 0
        for d in range(1, k):
            if ext[d] > ext[best]:
                best = d
        dims[s] = best
        x = pts[order[s], best]
        boxes[2 * s + 1] = (list(blo), bhi[:best] + [x] + bhi[best + 1:])
        boxes[2 * s + 2] = (blo[:best] + [x] + blo[best + 1:], list(bhi))
    return dims


def is_valid(pts, order, k, mode):
    n = len(order)
    dims = dims_of_arrangement(pts, order, k, mode)
    for i in range(1, n):
        child = i
        p = (i - 1) // 2
        while True:
            d = dims[p]
            if child == 2 * p + 1:
                if not strict_less(pts, order[i], order[p], d):
                    return False
            elif not strict_less(pts, order[p], order[i], d):
                return False
            if p == 0:
                break
            child, p = p, (p - 1) // 2
    return True


def tie_heavy(rng, n, k, values=(0.0, 1.0, 2.0)):
    return np.array([[rng.choice(values) for _ in range(k)] for _ in range(n)], dtype=np.float32)


# ------------------------------------------------------- paper's examples --
def test_fig1_six_points():
    pts, expected = fig1()
    out, orig = oracle.build(pts, k=2, mode=RR)
    np.testing.assert_array_equal(out, expected)
    np.testing.assert_array_equal(pts[orig], expected)


def test_sec5_walkthrough_final_array():
    blocks = walkthrough()
    _, _, _, x0, y0 = blocks[0]
    pts = np.array([x0, y0], dtype=np.float32).T.copy()
    out, _ = oracle.build(pts, k=2, mode=RR)
    step, _, _, xf, yf = blocks[-1]
    assert step == "final"
    np.testing.assert_array_equal(out[:, 0], np.array(xf, dtype=np.float32))
    np.testing.assert_array_equal(out[:, 1], np.array(yf, dtype=np.float32))


def test_sec5_walkthrough_every_step_of_the_level_loop():
    """The emulator of the paper's level loop reproduces every printed table
    (tags and coordinates after each sort and each tag update)."""
    blocks = walkthrough()
    _, _, _, x0, y0 = blocks[0]
    pts = np.array([x0, y0], dtype=np.float32).T.copy()
    seen = []

    def trace(step, l, tags, order):
        seen.append((step, l, list(tags), [int(pts[o, 0]) for o in order],
                     [int(pts[o, 1]) for o in order]))

    emulator.emulate(pts, 2, emulator.ROUND_ROBIN, trace)
    assert seen == [tuple(b) for b in blocks[1:]]


# ---------------------------------------------------------- brute force --
@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
def test_bruteforce_unique_valid_arrangement(mode):
    """Over all N! arrangements of tie-heavy inputs (N <= 7), exactly one
    satisfies the strict k-d condition, and it is the oracle's."""
    rng = random.Random(1234 + mode)
    cases = 0
    for n in range(1, 8):
        reps = 3 if n == 7 else 8
        for _ in range(reps):
            k = rng.randint(1, 3)
            pts = tie_heavy(rng, n, k) if rng.random() < 0.7 else \
                np.array([[rng.uniform(-3, 3) for _ in range(k)] for _ in range(n)], np.float32)
            valid = [p for p in itertools.permutations(range(n)) if is_valid(pts, p, k, mode)]
            assert len(valid) == 1, (n, k, pts)
            _, orig = oracle.build(pts, k, mode)
            assert tuple(int(o) for o in orig) == valid[0]
            cases += 1
    assert cases > 40


def test_bruteforce_n8_distinct():
    rng = random.Random(77)
    for mode in (RR, WIDEST, TIGHT):
        pts = np.array([[rng.uniform(0, 1) for _ in range(3)] for _ in range(8)], np.float32)
        valid = [p for p in itertools.permutations(range(8)) if is_valid(pts, p, 3, mode)]
        assert len(valid) == 1
        _, orig = oracle.build(pts, 3, mode)
        assert tuple(int(o) for o in orig) == valid[0]


# ------------------------------------------------------- closed forms --
def eytzinger(sorted_vals):
    n = len(sorted_vals)
    out = [None] * n
    it = iter(sorted_vals)

    def inorder(s):
        if s >= n:
            return
        inorder(2 * s + 1)
        out[s] = next(it)
        inorder(2 * s + 2)

    inorder(0)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 10, 31, 100, 257, 1000])
def test_k1_is_sorted_array_in_level_order(n):
    """k = 1: the tree is the sorted array laid out in level order (the
    textbook Eytzinger layout), for both split modes."""
    rng = np.random.default_rng(n)
    pts = rng.integers(0, max(2, n // 3), size=(n, 1)).astype(np.float32)
    ranked = sorted(range(n), key=lambda i: (fkey(pts[i, 0]), i))
    want = eytzinger(ranked)
    for mode in (RR, WIDEST, TIGHT):
        _, orig = oracle.build(pts, 1, mode)
        assert list(orig) == want


def test_subtree_size_counting_matches_recursive_definition():
    for n in range(0, 300):
        memo = {}

        def rec(s):
            if s >= n:
                return 0
            if s not in memo:
                memo[s] = 1 + rec(2 * s + 1) + rec(2 * s + 2)
            return memo[s]

        for s in range(n + 3):
            assert oracle.subtree_size(s, n) == rec(s)


def test_paper_ss_and_sb_formulas_match_counting():
    """Sec. 4.1 / 4.2 in O(1) equal the counted subtree size and the segment
    begin F(l) + sum of left siblings' sizes, for all s and N <= 1100."""
    for n in range(1, 1100):
        L = n.bit_length()
        for l in range(L):
            acc = (1 << l) - 1
            for s in range((1 << l) - 1, min(n, (1 << (l + 1)) - 1)):
                assert emulator.ss(s, n) == oracle.subtree_size(s, n)
                assert emulator.sb(s, l, n) == acc
                acc += oracle.subtree_size(s, n)


def test_literal_c_precedence_reading_of_ss_is_wrong():
    bad = sum(emulator.ss_literal(s, n) != oracle.subtree_size(s, n)
              for n in range(2, 300) for s in range(n))
    assert bad > 0


# ------------------------------------------------- algorithm agreement --
@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
def test_emulator_of_level_loop_matches_recursive_oracle(mode):
    rng = random.Random(99 + mode)
    for _ in range(300):
        n = rng.randint(1, 70)
        k = rng.randint(1, 4)
        if rng.random() < 0.5:
            pts = tie_heavy(rng, n, k, values=(-1.0, -0.0, 0.0, 0.5, 1.0))
        else:
            pts = np.array([[rng.gauss(0, 1) * (d + 1) for d in range(k)] for _ in range(n)],
                           np.float32)
        _, orig = oracle.build(pts, k, mode)
        assert list(emulator.emulate(pts, k, mode)) == list(orig)


# ------------------------------------------------------------ invariants --
@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
@pytest.mark.parametrize("gen", ["uniform", "mixed", "aniso"])
def test_checker_accepts_oracle_output_and_catches_planted_errors(mode, gen):
    n = 5000
    if gen == "uniform":
        pts = synth.uniform(n, 3, seed=5)
    elif gen == "mixed":
        pts = synth.mixed(n, 3, seed=6)
    else:
        pts = synth.aniso_float4(n, seed=7)
    out, orig = oracle.build(pts, 3, mode)
    assert oracle.check(pts, out, orig, 3, mode) == -1
    # the output is a permutation of the input
    assert sorted(orig.tolist()) == list(range(n))
    # planted: swap two nodes (records and indices together)
    o2, g2 = out.copy(), orig.copy()
    o2[[10, 2000]] = o2[[2000, 10]]
    g2[[10, 2000]] = g2[[2000, 10]]
    assert oracle.check(pts, o2, g2, 3, mode) >= 0
    # planted: a coordinate nudged by one ulp
    o3 = out.copy()
    o3[123, 0] = np.nextafter(o3[123, 0], np.float32(np.inf))
    assert oracle.check(pts, o3, orig, 3, mode) == 123
    # planted: index list that is not a permutation
    g4 = orig.copy()
    g4[5] = g4[6]
    assert oracle.check(pts, out, g4, 3, mode) >= 0


def test_perfect_tree_and_small_edge_sizes():
    for n in [0, 1, 2, 3, 4, 7, 15, 16, 17, 63, 64, 65]:
        pts = synth.uniform(n, 3, seed=n)
        out, orig = oracle.build(pts, 3, RR)
        assert oracle.check(pts, out, orig, 3, RR) == -1
        if n:
            assert sorted(orig.tolist()) == list(range(n))


def test_signed_zero_orders_below_positive_zero():
    pts = np.array([[0.0], [-0.0], [0.0]], dtype=np.float32)
    _, orig = oracle.build(pts, 1, RR)
    # strict order: (-0,1) < (+0,0) < (+0,2); root = rank ss(1) = 1 -> index 0
    assert list(orig) == [0, 1, 2]


def test_nan_is_rejected():
    pts = synth.uniform(50, 3, seed=1)
    pts[17, 2] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.build(pts, 3, RR)
    assert e.value.code == oracle.NAN_INPUT


def test_payload_moves_bytewise_and_is_never_compared():
    base = synth.uniform(3000, 3, seed=4)
    pts = synth.with_stride(base, 6)
    out, orig = oracle.build(pts, 3, RR)
    _, orig_plain = oracle.build(base, 3, RR)
    assert list(orig) == list(orig_plain)
    assert out.view(np.uint32).tobytes() == pts[orig].view(np.uint32).tobytes()


def test_widest_k1_equals_round_robin_and_dominant_axis_splits_first():
    pts = synth.uniform(500, 1, seed=2)
    assert list(oracle.build(pts, 1, WIDEST)[1]) == list(oracle.build(pts, 1, RR)[1])
    box = synth.aniso_float4(2000, seed=3)  # x extent 100, z 10, y 1
    out, orig = oracle.build(box, 3, WIDEST)
    xs = box[:, 0]
    # root splits x at the rank ss(1) element
    rank = sorted(range(2000), key=lambda i: (fkey(xs[i]), i))
    assert orig[0] == rank[oracle.subtree_size(1, 2000)]


def test_single_node_selector_matches_full_build():
    for mode in (RR, WIDEST, TIGHT):
        pts = synth.mixed(4000, 3, seed=11)
        _, orig = oracle.build(pts, 3, mode)
        rng = random.Random(mode)
        for s in [0, 1, 2, 3999] + [rng.randrange(4000) for _ in range(30)]:
            assert oracle.node(pts, 3, mode, s) == orig[s]


def test_tight_box_hand_example_and_difference_from_clipped_domain():
    """The hand-derived 7-point example (tests/golden/tight_box.txt): the
    tight-box rule and the clipped domain of Sec. 6 pick different dimensions
    at node 2, and each checker rejects the other rule's tree."""
    pts, want, want_clipped = tight_box()

    def as_orig(expected):
        return [next(i for i in range(len(pts)) if (pts[i] == row).all()) for row in expected]

    out, orig = oracle.build(pts, 2, TIGHT)
    assert list(orig) == as_orig(want)
    _, orig_c = oracle.build(pts, 2, WIDEST)
    assert list(orig_c) == as_orig(want_clipped)
    assert oracle.check(pts, out, orig, 2, TIGHT) == -1
    assert oracle.check(pts, out, orig, 2, WIDEST) >= 0
    out_c = pts[orig_c]
    assert oracle.check(pts, out_c, orig_c, 2, TIGHT) >= 0



# ------------------------------------------------------- int32 coordinates --
INT_EDGE = [-2**31, -2**31 + 1, -1, 0, 1, 2**24, 2**24 + 1, 2**31 - 2, 2**31 - 1]


def int_points(rng, n, k):
    """int32 coordinates with the extremes and pairs that float32 cannot tell
    apart (2^24 and 2^24 + 1; 2^31 - 2 and 2^31 - 1)."""
    return np.array([[rng.choice(INT_EDGE) for _ in range(k)] for _ in range(n)], dtype=np.int32)


def test_sec5_walkthrough_as_int2_points():
    """Sec. 5's points are int2: built as int32 coordinates the oracle gives the
    final array the paper prints, and the emulator every intermediate state."""
    blocks = walkthrough()
    _, _, _, x0, y0 = blocks[0]
    pts = np.array([x0, y0], dtype=np.int32).T.copy()
    out, orig = oracle.build(pts, 2, RR)
    _, _, _, xf, yf = blocks[-1]
    np.testing.assert_array_equal(out, np.array([xf, yf], dtype=np.int32).T)
    seen = []

    def trace(step, l, tags, order):
        seen.append((step, l, list(tags), [int(pts[o, 0]) for o in order],
                     [int(pts[o, 1]) for o in order]))

    emulator.emulate(pts, 2, RR, trace)
    assert seen == [tuple(b) for b in blocks[1:]]


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_int32_bruteforce_unique_valid_arrangement(mode):
    rng = random.Random(4321 + mode)
    for n in range(1, 8):
        for _ in range(4 if n == 7 else 8):
            k = rng.randint(1, 3)
            pts = int_points(rng, n, k)
            valid = [p for p in itertools.permutations(range(n)) if is_valid(pts, p, k, mode)]
            assert len(valid) == 1, (n, k, pts)
            _, orig = oracle.build(pts, k, mode)
            assert tuple(int(o) for o in orig) == valid[0]


@pytest.mark.parametrize("n", [1, 2, 7, 100, 1000])
def test_int32_k1_is_sorted_array_in_level_order(n):
    rng = random.Random(n)
    pts = int_points(rng, n, 1)
    ranked = sorted(range(n), key=lambda i: (int(pts[i, 0]), i))
    for mode in (RR, TIGHT):
        assert list(oracle.build(pts, 1, mode)[1]) == eytzinger(ranked)


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_int32_emulator_matches_oracle_and_checker(mode):
    rng = random.Random(55 + mode)
    for _ in range(150):
        n = rng.randint(1, 60)
        k = rng.randint(1, 3)
        pts = int_points(rng, n, k) if rng.random() < 0.5 else \
            np.array([[rng.randint(-50, 50) for _ in range(k)] for _ in range(n)], np.int32)
        out, orig = oracle.build(pts, k, mode)
        assert list(emulator.emulate(pts, k, mode)) == list(orig)
        assert oracle.check(pts, out, orig, k, mode) == -1
    # planted: a coordinate changed by one
    pts = synth_ints(5000, 3, seed=8)
    out, orig = oracle.build(pts, 3, mode)
    o2 = out.copy()
    o2[77, 1] += 1
    assert oracle.check(pts, o2, orig, 3, mode) >= 0


def synth_ints(n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-2**31, 2**31, size=(n, k), dtype=np.int64).astype(np.int32)


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_int32_equals_float32_on_values_both_represent_exactly(mode):
    """Integers below 2^24 in magnitude are exact in float32 and order the same
    way, so the int32 tree and the float32 tree of the same values agree."""
    rng = np.random.default_rng(9)
    ints = rng.integers(-2**24 + 1, 2**24, size=(3000, 3)).astype(np.int32)
    assert list(oracle.build(ints, 3, mode)[1]) == list(oracle.build(ints.astype(np.float32), 3, mode)[1])


def test_int32_with_the_clipped_domain_rule_is_refused():
    with pytest.raises(oracle.OracleError) as e:
        oracle.build(synth_ints(10, 3, seed=1), 3, WIDEST)
    assert e.value.code == oracle.INVALID


# ------------------------------------------------------ uint32 coordinates --
UINT_EDGE = [0, 1, 2**24, 2**24 + 1, 2**31 - 1, 2**31, 2**31 + 1, 2**32 - 2, 2**32 - 1]


def uint_points(rng, n, k):
    """uint32 coordinates on both sides of 2^31, where reading the bits as
    int32 would reverse the order."""
    return np.array([[rng.choice(UINT_EDGE) for _ in range(k)] for _ in range(n)], dtype=np.uint32)


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_uint32_bruteforce_unique_valid_arrangement(mode):
    rng = random.Random(8765 + mode)
    for n in range(1, 8):
        for _ in range(4 if n == 7 else 8):
            k = rng.randint(1, 3)
            pts = uint_points(rng, n, k)
            valid = [p for p in itertools.permutations(range(n)) if is_valid(pts, p, k, mode)]
            assert len(valid) == 1, (n, k, pts)
            _, orig = oracle.build(pts, k, mode)
            assert tuple(int(o) for o in orig) == valid[0]


@pytest.mark.parametrize("n", [1, 2, 7, 100, 1000])
def test_uint32_k1_is_sorted_array_in_level_order(n):
    rng = random.Random(100 + n)
    pts = uint_points(rng, n, 1)
    ranked = sorted(range(n), key=lambda i: (int(pts[i, 0]), i))  # int() of a uint32 is unsigned
    for mode in (RR, TIGHT):
        assert list(oracle.build(pts, 1, mode)[1]) == eytzinger(ranked)


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_uint32_equals_int32_with_the_top_bit_flipped(mode):
    """v -> v xor 2^31 maps the unsigned order of uint32 values onto the signed
    order of the int32 results and keeps every difference, so both trees (and
    both tight-box extents) agree."""
    rng = np.random.default_rng(12)
    u = rng.integers(0, 2**32, size=(3000, 3), dtype=np.uint64).astype(np.uint32)
    u[::7, 1] = np.uint32(2**31)  # ties on the boundary
    s = (u ^ np.uint32(0x80000000)).view(np.int32)
    assert list(oracle.build(u, 3, mode)[1]) == list(oracle.build(s, 3, mode)[1])


def test_uint32_tight_box_uses_unsigned_extents():
    """Three 2-D points A = (0, 0), B = (2^31 + 5, 1), C = (1, 2^31).  Unsigned
    extents: x spans 2^31 + 5, y spans 2^31, so the root splits in x, and the
    root is the x-rank-1 point (the left subtree of N = 3 holds one point):
    A < C < B in x, so C.  Read as int32, B's x and C's y are negative, y
    would span more (2^31 + 1 against 2^31 - 4) and the root would be A."""
    pts = np.array([[0, 0], [2**31 + 5, 1], [1, 2**31]], dtype=np.uint32)
    _, orig = oracle.build(pts, 2, TIGHT)
    assert list(orig) == [2, 0, 1]
    _, orig_signed = oracle.build(pts.view(np.int32), 2, TIGHT)
    assert orig_signed[0] == 0


@pytest.mark.parametrize("mode", [RR, TIGHT])
def test_uint32_emulator_matches_oracle_and_checker(mode):
    rng = random.Random(77 + mode)
    for _ in range(150):
        n = rng.randint(1, 60)
        k = rng.randint(1, 3)
        pts = uint_points(rng, n, k) if rng.random() < 0.5 else \
            np.array([[rng.randint(0, 60) for _ in range(k)] for _ in range(n)], np.uint32)
        out, orig = oracle.build(pts, k, mode)
        assert list(emulator.emulate(pts, k, mode)) == list(orig)
        assert oracle.check(pts, out, orig, k, mode) == -1
    # planted: the top bit of one coordinate flipped
    pts = np.random.default_rng(3).integers(0, 2**32, size=(5000, 3), dtype=np.uint64).astype(np.uint32)
    out, orig = oracle.build(pts, 3, mode)
    o2 = out.copy()
    o2[91, 0] ^= np.uint32(0x80000000)
    assert oracle.check(pts, o2, orig, 3, mode) >= 0


def test_uint32_refusals():
    pts = np.arange(30, dtype=np.uint32).reshape(10, 3)
    with pytest.raises(oracle.OracleError) as e:
        oracle.build(pts, 3, WIDEST)  # the clipped domain is float-only
    assert e.value.code == oracle.INVALID
    with pytest.raises(oracle.OracleError) as e:
        oracle.build(pts, 3, RR | oracle.INT32 | oracle.UINT32)
    assert e.value.code == oracle.INVALID


# ---- a subtree built on its own (the sharded single-tree build's local step)

def subtree_nodes(root, n):
    """Nodes of the subtree at `root` in its own level order."""
    out, first, width = [], root, 1
    while first < n:
        out += [t for t in range(first, min(first + width, n))]
        first, width = 2 * first + 1, 2 * width
    return out


def clipped_domain(out, k, node, scene_lo, scene_hi):
    """The domain of `node` in a clipped-domain tree `out` (records in level
    order): the scene box clipped by every ancestor's plane, the ancestors'
    dimensions recomputed top-down (float32 extents, lowest dimension wins
    ties) -- restated here from Sec. 6, independently of the oracle."""
    lo, hi = np.array(scene_lo, np.float32), np.array(scene_hi, np.float32)
    path = []
    v = node
    while v > 0:
        path.append(v)
        v = (v - 1) // 2
    p = 0
    for child in reversed(path):
        ext = [np.float32(hi[d]) - np.float32(lo[d]) for d in range(k)]
        d = 0
        for e in range(1, k):
            if ext[e] > ext[d]:
                d = e
        plane = out[p, d]
        if child == 2 * p + 1:
            hi[d] = plane
        else:
            lo[d] = plane
        p = child
    return np.concatenate([lo, hi])


def test_build_sub_at_the_root_is_the_whole_build():
    pts = synth.mixed(3000, 3, seed=12)
    for mode in (RR, WIDEST, TIGHT):
        dom = np.concatenate([pts.min(axis=0), pts.max(axis=0)]) if mode == WIDEST else None
        a, ao = oracle.build(pts, 3, mode)
        b, bo = oracle.build_sub(pts, 3, mode, 0, dom)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)) and np.array_equal(ao, bo)


@pytest.mark.parametrize("mode", [RR, WIDEST, TIGHT])
def test_build_sub_equals_the_subtrees_of_the_whole_build(mode):
    """Every subtree at depths 1..3 of a whole build, rebuilt on its own from
    its points in original-index order, is the same subtree: round robin from
    dimension depth mod k, the clipped-domain rule from the node's domain."""
    rng = np.random.default_rng(4 + mode)
    for n, k in ((2047, 3), (3001, 2), (777, 3), (100, 1)):
        pts = tie_heavy(random.Random(n), n, k, values=tuple(float(v) for v in range(9))) \
            if n == 777 else rng.random((n, k), dtype=np.float32)
        if mode == WIDEST:
            pts = pts * np.array([100.0, 1.0, 10.0][:k], np.float32)
        out, orig = oracle.build(pts, k, mode)
        for depth in (1, 2, 3):
            for node in range((1 << depth) - 1, (1 << (depth + 1)) - 1):
                if node >= n:
                    continue
                nodes = subtree_nodes(node, n)
                ids = np.sort(orig[nodes])
                dom = clipped_domain(out, k, node, pts.min(axis=0), pts.max(axis=0)) if mode == WIDEST else None
                sub, sorig = oracle.build_sub(pts[ids], k, mode, depth % k, dom)
                assert np.array_equal(ids[sorig], orig[nodes]), (n, k, node)
                assert np.array_equal(sub.view(np.uint32), out[nodes].view(np.uint32))


def test_build_sub_round_robin_is_the_build_of_rotated_coordinates():
    """Starting round robin at dimension f is the ordinary build of the
    coordinates rotated by f (column c holds dimension (c + f) mod k)."""
    pts = synth.uniform(1500, 3, seed=21)
    for f in range(3):
        rot = np.ascontiguousarray(np.roll(pts, -f, axis=1))
        _, want = oracle.build(rot, 3, RR)
        _, got = oracle.build_sub(pts, 3, RR, f)
        assert np.array_equal(want, got)
    with pytest.raises(oracle.OracleError):
        oracle.build_sub(pts, 3, RR, 3)
    with pytest.raises(oracle.OracleError):
        oracle.build_sub(pts, 3, WIDEST, 0, None)
