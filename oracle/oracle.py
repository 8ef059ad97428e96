"""ctypes wrapper around ``kd_oracle.c`` (test infrastructure only).

The C file is the oracle: the plain recursive sort-split-recurse builder that
Observation 1 (Sec. 2.1) defines, a strict invariant checker, and a one-node
path selector for sampled checks at sizes where the full build is slow.  This
module compiles it with gcc on first use (or when ``compile_oracle()`` is
called from the build step) and exposes numpy-level functions.

Records are passed as 2-D C-contiguous numpy arrays with 4-byte items (one row
per record, row bytes = stride); the first ``k`` columns are the coordinates
and any further columns are payload that is moved, never compared.  An int32
or uint32 array has int32 or uint32 coordinates (the oracle's INT32 / UINT32
mode flag is set from the dtype unless the mode already carries one); any
other 4-byte dtype is read as float32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

ROUND_ROBIN = 0
WIDEST = 1
WIDEST_TIGHT = 2  # widest side of the subtree's own (tight) bounding box
INT32 = 0x100     # mode flag: int32 coordinates
UINT32 = 0x200    # mode flag: uint32 coordinates

OK = 0
INVALID = 1
NOMEM = 2
NAN_INPUT = 4
NOT_KD = 6

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libkd_oracle.so")
_lock = threading.Lock()
_lib = None


def compile_oracle(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no -march flags, so the same
    source builds on x86-64 and aarch64).  Returns the library path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(compile_oracle())
            i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.kdo_build.argtypes = [vp, i64, i32, i32, i32, vp, vp]
            lib.kdo_build.restype = i32
            lib.kdo_check.argtypes = [vp, vp, vp, i64, i32, i32, i32, ctypes.POINTER(i64)]
            lib.kdo_check.restype = i32
            lib.kdo_node.argtypes = [vp, i64, i32, i32, i32, i64, ctypes.POINTER(ctypes.c_int32)]
            lib.kdo_node.restype = i32
            lib.kdo_build_sub.argtypes = [vp, i64, i32, i32, i32, i32, vp, vp, vp]
            lib.kdo_build_sub.restype = i32
            lib.kdo_subtree_size.argtypes = [i64, i64]
            lib.kdo_subtree_size.restype = i64
            _lib = lib
    return _lib


def _records(points: np.ndarray) -> np.ndarray:
    if points.ndim != 2 or points.dtype.itemsize != 4:
        raise ValueError("records must be a 2-D array of 4-byte items")
    return np.ascontiguousarray(points)


def _mode(points: np.ndarray, mode: int) -> int:
    if mode & (INT32 | UINT32):
        return mode
    return mode | {np.dtype(np.int32): INT32, np.dtype(np.uint32): UINT32}.get(points.dtype, 0)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} returned {code}")
        self.code = code


def build(points: np.ndarray, k: int, mode: int = ROUND_ROBIN):
    """Returns (records in level order, original index of each node)."""
    pts = _records(points)
    n, w = pts.shape
    out = np.empty_like(pts)
    orig = np.empty(n, dtype=np.int32)
    rc = _load().kdo_build(pts.ctypes.data, n, k, 4 * w, _mode(pts, mode), out.ctypes.data,
                           orig.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "kdo_build")
    return out, orig


def build_sub(points: np.ndarray, k: int, mode: int = ROUND_ROBIN, first_dim: int = 0, root_domain=None):
    """The subtree below a node of a larger tree, built on its own: round
    robin starts at dimension ``first_dim``; the clipped-domain rule starts
    from ``root_domain`` (k lower bounds, then k upper bounds).  Returns
    (records in the subtree's level order, position of each node's record)."""
    pts = _records(points)
    n, w = pts.shape
    out = np.empty_like(pts)
    orig = np.empty(n, dtype=np.int32)
    dom = None if root_domain is None else np.ascontiguousarray(root_domain, dtype=np.float32)
    rc = _load().kdo_build_sub(pts.ctypes.data, n, k, 4 * w, _mode(pts, mode), first_dim,
                               None if dom is None else dom.ctypes.data, out.ctypes.data, orig.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "kdo_build_sub")
    return out, orig


def check(in_points: np.ndarray, out_points: np.ndarray, orig: np.ndarray, k: int,
          mode: int = ROUND_ROBIN) -> int:
    """First node violating permutation / strict k-d invariants, or -1."""
    a = _records(in_points)
    b = _records(out_points)
    o = np.ascontiguousarray(orig, dtype=np.int32)
    if a.shape != b.shape or o.shape != (a.shape[0],):
        raise ValueError("shape mismatch")
    bad = ctypes.c_int64(-1)
    rc = _load().kdo_check(a.ctypes.data, b.ctypes.data, o.ctypes.data, a.shape[0], k,
                           4 * a.shape[1], _mode(a, mode), ctypes.byref(bad))
    if rc not in (OK, NOT_KD):
        raise OracleError(rc, "kdo_check")
    return int(bad.value)


def node(points: np.ndarray, k: int, mode: int, s: int) -> int:
    """Original index of the record that belongs at node ``s``."""
    pts = _records(points)
    out = ctypes.c_int32(-1)
    rc = _load().kdo_node(pts.ctypes.data, pts.shape[0], k, 4 * pts.shape[1], _mode(pts, mode), s,
                          ctypes.byref(out))
    if rc != OK:
        raise OracleError(rc, "kdo_node")
    return int(out.value)


def subtree_size(s: int, n: int) -> int:
    return int(_load().kdo_subtree_size(s, n))
