"""Thin Python binding of the C ABI in ``include/kdb.h``.

Argument marshalling only: every step of the build runs in the CUDA library
``_build/libkdb.so``.  Device buffers are torch CUDA tensors (PyTorch provides
device memory and streams); the functions take the tensor's data pointer and
the current torch stream.  There is no fallback: if the library has not been
built, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

ROUND_ROBIN = 0
WIDEST_EXTENT = 1
WIDEST_TIGHT = 2  # widest side of the subtree's own bounding box (k <= 3)
COORDS_INT32 = 0x100  # mode flag: int32 coordinates (set from an int32 tensor's dtype)
COORDS_UINT32 = 0x200  # mode flag: uint32 coordinates (set from a uint32 tensor's dtype)

OK = 0
ERR_INVALID_ARGUMENT = 1
ERR_OUT_OF_MEMORY = 2
ERR_CUDA = 3
ERR_NAN_INPUT = 4
ERR_TIMEOUT = 5
ERR_NOT_A_KD_TREE = 6
ERR_INTERNAL = 7

PLACEMENT_AUTO = 0
MEMORY_AUTO, MEMORY_FAST, MEMORY_LEAN = 0, 1, 2
PLACEMENT_IN_PLACE = 1

TUNE_PARTITION = 0
TUNE_RADIX = 1
TUNE_DIGITS = 2

FAULT_NONE = 0
FAULT_ALLOC = 1
FAULT_LOOKBACK = 2
FAULT_LOOKBACK_PARTITION = 3
FAULT_LOW_MEMORY = 4

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkdb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "kdb.h")

_lib = None
_lock = threading.Lock()


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_inflight_batches", ctypes.c_int),
                ("max_batch_requests", ctypes.c_int), ("max_batch_points", ctypes.c_int64)]


class RequestResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("n", ctypes.c_int64),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("submitted", "completed", "failed", "batches", "retried_alone",
                 "max_batch_requests", "max_inflight_batches", "queued", "inflight_requests")] + \
               [(f, ctypes.c_size_t) for f in ("budget_bytes", "used_bytes", "max_used_bytes")]


class Tuning(ctypes.Structure):
    _fields_ = [("partition_shape", ctypes.c_int32), ("radix_shape", ctypes.c_int32),
                ("digit_bits", ctypes.c_int32)]


class KdbError(RuntimeError):
    def __init__(self, code: int, call: str):
        super().__init__(f"{call}: {status_string(code)} ({code})")
        self.code = code


def declared_symbols() -> list[str]:
    """Names of the entry points declared in include/kdb.h."""
    with open(HEADER) as f:
        text = f.read()
    return re.findall(r"KDB_API\s+[\w\s\*]+?\b(kdb_\w+)\s*\(", text)


def load():
    """Loads the CUDA library; raises if it was not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        sig = {
            "kdb_status_string": ([i32], ctypes.c_char_p),
            "kdb_version": ([], i32),
            "kdb_build": ([vp, i64, i32, i32, i32, vp], i32),
            "kdb_workspace_size": ([i64, i32, i32, i32], sz),
            "kdb_build_ex": ([vp, i64, i32, i32, i32, vp, sz, vp, vp, vp], i32),
            "kdb_build_batched": ([vp, vp, i32, i32, i32, i32, vp], i32),
            "kdb_build_host": ([vp, i64, i32, i32, i32, vp], i32),
            "kdb_build_noalloc": ([vp, i64, i32, i32, i32, vp], i32),
            "kdb_validate": ([vp, i64, i32, i32, i32, ctypes.POINTER(i64), vp], i32),
            "kdb_debug_inject_fault": ([i32, i64], i32),
            "kdb_set_placement": ([i32], i32),
            "kdb_set_memory_mode": ([i32], i32),
            "kdb_lean_workspace_size": ([i64, i32, i32, i32], sz),
            "kdb_tuning_shape_count": ([i32], i32),
            "kdb_tuning_shape": ([i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                  ctypes.POINTER(i32)], i32),
            "kdb_get_tuning": ([ctypes.POINTER(Tuning)], i32),
            "kdb_set_tuning": ([ctypes.POINTER(Tuning)], i32),
            "kdb_lookup_tuning": ([i64, i32, i32, i32, ctypes.POINTER(Tuning), ctypes.POINTER(i32)], i32),
            "kdb_clear_tuning_table": ([], None),
            "kdb_save_tuning": ([ctypes.c_char_p], i32),
            "kdb_load_tuning": ([ctypes.c_char_p], i32),
            "kdb_autotune": ([vp, i64, i32, i32, i32, i32, ctypes.POINTER(Tuning),
                              ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), vp], i32),
            "kdb_plan_create": ([vp, i32, i32, i32, i32, ctypes.POINTER(vp)], i32),
            "kdb_plan_enqueue": ([vp, vp, vp], i32),
            "kdb_plan_status": ([vp, vp], i32),
            "kdb_plan_workspace_bytes": ([vp], sz),
            "kdb_plan_destroy": ([vp], None),
            "kdb_profile_start": ([], None),
            "kdb_profile_stop": ([ctypes.POINTER(KernelStat), i32], i32),
            "kdb_launch_count": ([], i64),
            "kdb_batched_workspace_size": ([vp, i32, i32, i32, i32], sz),
            "kdb_build_batched_async": ([vp, vp, i32, i32, i32, i32, vp, sz, vp, vp], i32),
            "kdb_error_word_status": ([ctypes.c_uint32], i32),
            "kdb_server_create": ([ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)], i32),
            "kdb_server_submit": ([vp, vp, vp, i64, i32, i32, i32, ctypes.POINTER(i64)], i32),
            "kdb_server_poll": ([vp, ctypes.POINTER(RequestResult), i32, i32], i32),
            "kdb_server_get_stats": ([vp, ctypes.POINTER(ServerStats)], i32),
            "kdb_server_destroy": ([vp], i32),
            "kdb_build_subtree": ([vp, i64, i32, i32, i32, i32, vp, vp, vp], i32),
            "kdb_dist_histogram": ([vp, i64, i32, i32, i32, vp, i32, vp, vp, i32, ctypes.c_uint32, vp, vp], i32),
            "kdb_dist_box": ([vp, i64, i32, i32, i32, vp, i32, vp, vp], i32),
            "kdb_dist_assign": ([vp, i64, i32, i32, i32, vp, i32, vp, vp, ctypes.c_uint32, vp, vp], i32),
            "kdb_dist_partition": ([vp, i64, i32, vp, i32, i32, ctypes.c_uint32, vp, vp,
                                    ctypes.POINTER(i64), vp], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def status_string(code: int) -> str:
    try:
        return load().kdb_status_string(code).decode()
    except Exception:  # library not loadable: still give a message
        return f"status {code}"


def _stream(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _records(points):
    """(pointer, n, stride_bytes) of a 2-D contiguous tensor of 4-byte items."""
    if points.dim() != 2 or points.element_size() != 4 or not points.is_contiguous():
        raise ValueError("points must be a contiguous 2-D tensor of 4-byte items (one row per record)")
    return points.data_ptr(), points.shape[0], 4 * points.shape[1]


def _mode(points, mode: int) -> int:
    """The mode argument: the split rule, plus COORDS_INT32 / COORDS_UINT32 for
    int32 / uint32 records unless the mode already names a coordinate type
    (so that uint32 data can also be passed as an int32 view)."""
    import torch

    if mode & (COORDS_INT32 | COORDS_UINT32):
        return mode
    if points.dtype == torch.int32:
        return mode | COORDS_INT32
    if points.dtype == getattr(torch, "uint32", None):
        return mode | COORDS_UINT32
    return mode


def _check(rc: int, call: str):
    if rc != OK:
        raise KdbError(rc, call)


def kdb_version() -> int:
    return load().kdb_version()


def kdb_status_string(code: int) -> str:
    return status_string(code)


def kdb_build(points, k: int, mode: int = ROUND_ROBIN, stream=None) -> None:
    """Permutes the CUDA tensor ``points`` (rows = records, first k columns
    float32 coordinates) in place into a left-balanced k-d tree."""
    ptr, n, stride = _records(points)
    _check(load().kdb_build(ptr, n, k, stride, _mode(points, mode), _stream(stream)), "kdb_build")


def kdb_workspace_size(n: int, k: int, stride_bytes: int, mode: int = ROUND_ROBIN) -> int:
    return int(load().kdb_workspace_size(n, k, stride_bytes, mode))


def kdb_build_ex(points, k: int, mode: int = ROUND_ROBIN, workspace=None, out_orig_index=None,
                 out_split_dim=None, stream=None) -> None:
    ptr, n, stride = _records(points)
    ws = workspace.data_ptr() if workspace is not None else None
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    oi = out_orig_index.data_ptr() if out_orig_index is not None else None
    od = out_split_dim.data_ptr() if out_split_dim is not None else None
    _check(load().kdb_build_ex(ptr, n, k, stride, _mode(points, mode), ws, wsb, oi, od,
                               _stream(stream)), "kdb_build_ex")


def kdb_build_batched(points, offsets, k: int, mode: int = ROUND_ROBIN, stream=None) -> None:
    """``offsets``: sequence of num_sets+1 record offsets (host)."""
    ptr, n, stride = _records(points)
    offs = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
    if offs[len(offsets) - 1] != n:
        raise ValueError("offsets must end at the number of records")
    _check(load().kdb_build_batched(ptr, offs, len(offsets) - 1, k, stride, _mode(points, mode),
                                    _stream(stream)), "kdb_build_batched")


def kdb_build_host(points, k: int, mode: int = ROUND_ROBIN, stream=None) -> None:
    """``points``: host (CPU, ideally pinned) tensor, permuted in place."""
    ptr, n, stride = _records(points)
    _check(load().kdb_build_host(ptr, n, k, stride, _mode(points, mode), _stream(stream)),
           "kdb_build_host")


def kdb_build_subtree(points, k: int, mode: int = ROUND_ROBIN, first_dim: int = 0, root_domain=None,
                      out_orig_index=None, stream=None) -> None:
    """kdb_build of the subtree below one node of a larger tree: round robin
    continues from ``first_dim``; the clipped-domain rule starts from
    ``root_domain`` (2k floats: lower corner, then upper corner)."""
    ptr, n, stride = _records(points)
    dom = None
    if root_domain is not None:
        vals = [float(v) for v in root_domain]
        dom = (ctypes.c_float * len(vals))(*vals)
    oi = out_orig_index.data_ptr() if out_orig_index is not None else None
    _check(load().kdb_build_subtree(ptr, n, k, stride, _mode(points, mode), first_dim, dom, oi,
                                    _stream(stream)), "kdb_build_subtree")


def kdb_dist_histogram(points, k: int, mode: int, tags, level: int, node_dim, node_prefix, prefix_bits: int,
                       index_base: int, hist, stream=None) -> None:
    """Radix-select digit histograms of one top level of a sharded build
    (device tensors: tags int32[n], node_dim uint8[2^level], node_prefix
    int64[2^level], hist int32[2^level, 256])."""
    ptr, n, stride = _records(points)
    _check(load().kdb_dist_histogram(ptr, n, k, stride, _mode(points, mode), tags.data_ptr(), level,
                                     node_dim.data_ptr(), node_prefix.data_ptr(), prefix_bits, index_base,
                                     hist.data_ptr(), _stream(stream)), "kdb_dist_histogram")


def kdb_dist_box(points, k: int, mode: int, tags, level: int, box, stream=None) -> None:
    """Per node of one top level: min and max coordinate keys (box int32[2^level, 2k])."""
    ptr, n, stride = _records(points)
    _check(load().kdb_dist_box(ptr, n, k, stride, _mode(points, mode), tags.data_ptr(), level, box.data_ptr(),
                               _stream(stream)), "kdb_dist_box")


def kdb_dist_assign(points, k: int, mode: int, tags, level: int, node_dim, pivot, index_base: int, pinned,
                    stream=None) -> None:
    """Tag update of one top level against the nodes' pivot keys (pivot
    int64[2^level]); pinned int64[2^level] receives the local position of
    each pivot held here."""
    ptr, n, stride = _records(points)
    _check(load().kdb_dist_assign(ptr, n, k, stride, _mode(points, mode), tags.data_ptr(), level,
                                  node_dim.data_ptr(), pivot.data_ptr(), index_base, pinned.data_ptr(),
                                  _stream(stream)), "kdb_dist_assign")


def kdb_dist_partition(points, tags, first_node: int, num_dest: int, index_base: int, out_points, out_index,
                       stream=None) -> list:
    """Stable partition of the points by destination tag - first_node; returns
    the record count of each destination."""
    ptr, n, stride = _records(points)
    counts = (ctypes.c_int64 * num_dest)()
    _check(load().kdb_dist_partition(ptr, n, stride, tags.data_ptr(), first_node, num_dest, index_base,
                                     out_points.data_ptr(), out_index.data_ptr(), counts, _stream(stream)),
           "kdb_dist_partition")
    return [int(c) for c in counts]


NOALLOC_MAX_POINTS = 262144
NOALLOC_SCRATCH_BYTES = 64 << 20  # the static workspace array (KDB_NOALLOC_SCRATCH_BYTES)


def kdb_build_noalloc(points, k: int, mode: int = ROUND_ROBIN, stream=None) -> None:
    """kdb_build whose workspace is the library's static device array: for
    callers that cannot allocate device memory when they build.  At most
    NOALLOC_MAX_POINTS records; calls must not overlap on the GPU."""
    ptr, n, stride = _records(points)
    _check(load().kdb_build_noalloc(ptr, n, k, stride, _mode(points, mode), _stream(stream)),
           "kdb_build_noalloc")


def kdb_validate(points, k: int, mode: int = ROUND_ROBIN, stream=None) -> int:
    """Returns -1 if ``points`` is a valid k-d tree, else the first bad node."""
    ptr, n, stride = _records(points)
    bad = ctypes.c_int64(-1)
    rc = load().kdb_validate(ptr, n, k, stride, _mode(points, mode), ctypes.byref(bad), _stream(stream))
    if rc not in (OK, ERR_NOT_A_KD_TREE):
        raise KdbError(rc, "kdb_validate")
    return int(bad.value)


class Plan:
    """A build prepared once (kdb_plan_create) and enqueued many times; the
    enqueue is capture-safe (CUDA graphs).  ``offsets``: record offsets of the
    sets (num_sets + 1 entries), or a single point count."""

    def __init__(self, offsets, k: int, stride_bytes: int, mode: int = ROUND_ROBIN):
        if isinstance(offsets, int):
            offsets = [0, offsets]
        self.offsets = [int(o) for o in offsets]
        offs = (ctypes.c_int64 * len(self.offsets))(*self.offsets)
        h = ctypes.c_void_p()
        _check(load().kdb_plan_create(offs, len(self.offsets) - 1, k, stride_bytes, mode,
                                      ctypes.byref(h)), "kdb_plan_create")
        self._h = h
        self.k, self.stride, self.mode = k, stride_bytes, mode

    def enqueue(self, points, stream=None) -> None:
        ptr, n, stride = _records(points)
        if n != self.offsets[-1] or stride != self.stride:
            raise ValueError("points do not match the plan's layout")
        _check(load().kdb_plan_enqueue(self._h, ptr, _stream(stream)), "kdb_plan_enqueue")

    def status(self, stream=None) -> None:
        _check(load().kdb_plan_status(self._h, _stream(stream)), "kdb_plan_status")

    @property
    def workspace_bytes(self) -> int:
        return int(load().kdb_plan_workspace_bytes(self._h))

    def close(self) -> None:
        if self._h:
            load().kdb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kdb_batched_workspace_size(offsets, k: int, stride_bytes: int, mode: int = ROUND_ROBIN) -> int:
    offs = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
    return int(load().kdb_batched_workspace_size(offs, len(offsets) - 1, k, stride_bytes, mode))


def kdb_build_batched_async(points, offsets, k: int, mode: int, workspace, error_word,
                            stream=None) -> None:
    """Enqueues a batched build with caller workspace (CUDA uint8 tensor) and a
    device error word (CUDA int32 tensor of one element, or None)."""
    ptr, n, stride = _records(points)
    offs = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
    if offs[len(offsets) - 1] != n:
        raise ValueError("offsets must end at the number of records")
    ew = error_word.data_ptr() if error_word is not None else None
    _check(load().kdb_build_batched_async(ptr, offs, len(offsets) - 1, k, stride, _mode(points, mode),
                                          workspace.data_ptr(),
                                          workspace.numel() * workspace.element_size(), ew,
                                          _stream(stream)), "kdb_build_batched_async")


def kdb_error_word_status(word: int) -> int:
    return int(load().kdb_error_word_status(word & 0xFFFFFFFF))


class Server:
    """The library's build server (kdb_server_*): requests are submitted as
    host tensors and built on the current device by continuous batching.
    Keeps a reference to each request's tensors until its result is polled."""

    def __init__(self, budget_bytes: int, max_inflight_batches: int = 3,
                 max_batch_requests: int = 4096, max_batch_points: int = 1 << 26):
        cfg = ServerConfig(int(budget_bytes), int(max_inflight_batches), int(max_batch_requests),
                           int(max_batch_points))
        h = ctypes.c_void_p()
        _check(load().kdb_server_create(ctypes.byref(cfg), ctypes.byref(h)), "kdb_server_create")
        self._h = h
        self._keep = {}
        self._res = (RequestResult * 256)()

    def submit(self, points, k: int, mode: int = ROUND_ROBIN, out=None) -> int:
        """``points``: CPU tensor (rows = records; pinned for asynchronous
        copies); ``out``: CPU tensor of the same shape for the tree, or None
        to build in place."""
        if points.is_cuda:
            raise ValueError("Server.submit takes host tensors")
        ptr, n, stride = _records(points)
        dst = points if out is None else out
        if dst.shape != points.shape or dst.dtype != points.dtype or not dst.is_contiguous():
            raise ValueError("out must be a contiguous tensor shaped like points")
        rid = ctypes.c_int64(-1)
        _check(load().kdb_server_submit(self._h, ptr, dst.data_ptr(), n, k, stride,
                                        _mode(points, mode), ctypes.byref(rid)), "kdb_server_submit")
        self._keep[rid.value] = (points, dst)
        return int(rid.value)

    def poll(self, timeout_ms: int = 0, max_results: int = 256) -> list[dict]:
        m = min(max_results, len(self._res))
        n = load().kdb_server_poll(self._h, self._res, m, int(timeout_ms))
        if n < 0:
            raise KdbError(ERR_INVALID_ARGUMENT, "kdb_server_poll")
        out = []
        for i in range(n):
            r = self._res[i]
            self._keep.pop(int(r.id), None)
            out.append({"id": int(r.id), "status": int(r.status), "n": int(r.n),
                        "submit_s": r.submit_s, "admit_s": r.admit_s, "done_s": r.done_s})
        return out

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().kdb_server_get_stats(self._h, ctypes.byref(st)), "kdb_server_get_stats")
        return {f: int(getattr(st, f)) for f, _ in ServerStats._fields_}

    def close(self) -> None:
        if self._h:
            rc = load().kdb_server_destroy(self._h)
            self._h = None
            self._keep.clear()
            _check(rc, "kdb_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kdb_set_memory_mode(mode: int) -> int:
    """Process-wide memory mode (MEMORY_AUTO / MEMORY_FAST / MEMORY_LEAN) of
    kdb_build; returns the previous one."""
    return load().kdb_set_memory_mode(mode)


def kdb_lean_workspace_size(n: int, k: int, stride_bytes: int, mode: int = ROUND_ROBIN) -> int:
    """Device bytes of the memory-lean build (0: invalid arguments or n < 4)."""
    return int(load().kdb_lean_workspace_size(n, k, stride_bytes, mode))


def kdb_set_placement(placement: int) -> int:
    """Process-wide placement setting (PLACEMENT_AUTO / PLACEMENT_IN_PLACE);
    returns the previous one."""
    return load().kdb_set_placement(placement)


def kdb_tuning_shapes(kernel: int) -> list[tuple[int, int, int]]:
    """(threads, items per thread, blocks per SM) of each compiled shape of
    ``kernel`` (TUNE_PARTITION or TUNE_RADIX); for TUNE_DIGITS (bits, passes
    per key, 1) of each compiled digit width."""
    lib = load()
    count = lib.kdb_tuning_shape_count(kernel)
    if count < 0:
        raise KdbError(ERR_INVALID_ARGUMENT, "kdb_tuning_shape_count")
    out = []
    for i in range(count):
        t, it, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.kdb_tuning_shape(kernel, i, ctypes.byref(t), ctypes.byref(it), ctypes.byref(b)),
               "kdb_tuning_shape")
        out.append((t.value, it.value, b.value))
    return out


def kdb_digit_widths() -> list[int]:
    """The compiled digit widths of the level-0 sort, in bits."""
    return [w for w, _, _ in kdb_tuning_shapes(TUNE_DIGITS)]


def kdb_get_tuning() -> tuple[int, int, int]:
    """Process-wide (partition shape, radix shape, digit bits)."""
    t = Tuning()
    _check(load().kdb_get_tuning(ctypes.byref(t)), "kdb_get_tuning")
    return t.partition_shape, t.radix_shape, t.digit_bits


def kdb_set_tuning(partition_shape: int, radix_shape: int, digit_bits: int = 8) -> None:
    t = Tuning(partition_shape, radix_shape, digit_bits)
    _check(load().kdb_set_tuning(ctypes.byref(t)), "kdb_set_tuning")


def kdb_lookup_tuning(n: int, k: int, stride_bytes: int, mode: int = ROUND_ROBIN):
    """The setting a build of this kind takes: ((partition shape, radix
    shape, digit bits), whether it comes from the tuning table).  ``mode`` is
    the mode argument as the build passes it (coordinate-type flags
    included)."""
    t = Tuning()
    hit = ctypes.c_int32()
    _check(load().kdb_lookup_tuning(n, k, stride_bytes, mode, ctypes.byref(t), ctypes.byref(hit)),
           "kdb_lookup_tuning")
    return (t.partition_shape, t.radix_shape, t.digit_bits), bool(hit.value)


def kdb_clear_tuning_table() -> None:
    load().kdb_clear_tuning_table()


def kdb_save_tuning(path: str) -> None:
    """Writes the process-wide setting and the tuning table to a JSON file."""
    _check(load().kdb_save_tuning(os.fsencode(path)), "kdb_save_tuning")


def kdb_load_tuning(path: str) -> None:
    """Replaces the process-wide setting and the tuning table with a file
    written by kdb_save_tuning."""
    _check(load().kdb_load_tuning(os.fsencode(path)), "kdb_load_tuning")


def kdb_autotune(points, k: int, mode: int = ROUND_ROBIN, reps: int = 3, stream=None) -> dict:
    """Times every (partition shape, radix shape, digit width) on a copy of
    ``points`` and keeps the fastest as the process-wide setting and as the
    table entry of this kind of build.  Returns {"best": (p, r, bits),
    "best_ms": median ms, "ms": {(p, r, bits): median ms}} (choices not timed
    are left out)."""
    ptr, n, stride = _records(points)
    lib = load()
    npart = lib.kdb_tuning_shape_count(TUNE_PARTITION)
    nrad = lib.kdb_tuning_shape_count(TUNE_RADIX)
    widths = kdb_digit_widths()
    nw = len(widths)
    best = Tuning()
    best_ms = ctypes.c_float()
    ms = (ctypes.c_float * (npart * nrad * nw))()
    _check(lib.kdb_autotune(ptr, n, k, stride, _mode(points, mode), reps, ctypes.byref(best),
                            ctypes.byref(best_ms), ms, _stream(stream)), "kdb_autotune")
    table = {(c // (nrad * nw), (c // nw) % nrad, widths[c % nw]): ms[c]
             for c in range(npart * nrad * nw) if ms[c] >= 0}
    return {"best": (best.partition_shape, best.radix_shape, best.digit_bits), "best_ms": best_ms.value,
            "ms": table}


def kdb_debug_inject_fault(fault: int, arg: int = 0) -> int:
    return load().kdb_debug_inject_fault(fault, arg)


def kdb_profile_start() -> None:
    load().kdb_profile_start()


def kdb_profile_stop() -> list[dict]:
    """Per kernel kind: launches, summed device ms, summed algorithmic bytes."""
    buf = (KernelStat * 16)()
    n = load().kdb_profile_stop(buf, 16)
    if n < 0:
        raise KdbError(ERR_CUDA, "kdb_profile_stop")
    return [{"name": buf[i].name.decode(), "launches": int(buf[i].launches), "ms": buf[i].ms,
             "bytes": buf[i].bytes} for i in range(n)]


def kdb_launch_count() -> int:
    return int(load().kdb_launch_count())
