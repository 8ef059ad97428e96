"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


def walkthrough():
    """List of (step, l, tags, x, y) blocks of the Sec. 5 example."""
    lines = list(_lines("walkthrough_sec5.txt"))
    blocks = []
    for i in range(0, len(lines), 4):
        step, l = lines[i].split()
        rows = {}
        for ln in lines[i + 1:i + 4]:
            name, *vals = ln.split()
            rows[name] = [int(v) for v in vals]
        blocks.append((step, int(l), rows["tags"], rows["x"], rows["y"]))
    return blocks


def fig1():
    d = {}
    for ln in _lines("fig1.txt"):
        name, *pts = ln.split()
        d[name] = np.array([[float(c) for c in p.split(",")] for p in pts], dtype=np.float32)
    return d["input"], d["expected"]


def tight_box():
    """The hand-derived tight-box example: (input, expected, expected with the
    clipped domain of Sec. 6)."""
    d = {}
    for ln in _lines("tight_box.txt"):
        name, *pts = ln.split()
        d[name] = np.array([[float(c) for c in p.split(",")] for p in pts], dtype=np.float32)
    return d["input"], d["expected"], d["expected_clipped"]
