"""Benchmark of the GB300 k-d tree build.

One step = one complete build (every level of the method plus the final
placement) of one synthetic point set already resident in device memory.
Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
plain recursive builder the parity tests compare against) on a bounded
sample of the same workload.

Launch: ``python bench.py [--gpus 1] [--steps K] [--warmup W]``; for N > 1 under
``torch.distributed.run`` each rank builds its own replica of the workload
(a single tree does not shard) and rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2211_00120_gb300 import synth  # noqa: E402

METRIC = "Mpts/s k-d build at 1e8 float3, % of HBM roofline; batched vs serial builds/s"

WORKLOADS = {
    # name: (description, n, k, stride floats, split mode, generator)
    "uniform_1e8_f3_rr": ("1e8 float3 points, uniform [0,1)^3 (seed 0), round-robin split",
                          100_000_000, 3, 3, 0, lambda n: synth.uniform(n, 3, seed=0)),
    "mixed_1e7_f3_rr": ("1e7 float3 points, half uniform, half 64 Gaussian clusters (sigma 0.01), "
                        "1% exact duplicates (seed 1), round-robin split",
                        10_000_000, 3, 3, 0, lambda n: synth.mixed(n, 3, seed=1)),
    "aniso_1e8_f4_widest": ("1e8 float4 points (xyz + payload) uniform in [0,100)x[0,1)x[0,10) "
                            "(seed 2), widest-extent split",
                            100_000_000, 3, 4, 1, lambda n: synth.aniso_float4(n, seed=2)),
    "int1_1e8_rr": ("1e8 int32 points, k = 1 (the paper's int1 data), uniform over the int32 "
                    "range (seed 0), round-robin split",
                    100_000_000, 1, 1, 0, lambda n: synth.int32_uniform(n, 1, seed=0)),
    "aniso_1e8_f4_tight": ("1e8 float4 points (xyz + payload) uniform in [0,100)x[0,1)x[0,10) "
                           "(seed 2), widest side of each subtree's tight box",
                           100_000_000, 3, 4, 2, lambda n: synth.aniso_float4(n, seed=2)),
}
# algorithmic bytes per item of each kernel kind (matches the library's
# profiling counters): used to turn a launch's bytes into items
BYTES_PER_ITEM = {"partition_pass": 32.0, "radix_pass": 32.0}


# the source file that defines each kernel kind of the k <= 3 path
KIND_SOURCE = {"partition_pass": "kdb_part.cu", "radix_pass": "kdb_lists.cu",
               "pivots": "kdb_part.cu", "build_lists": "kdb_lists.cu",
               "local_finish": "kdb_local.cu", "placement": "kdb_tree.cu",
               "prepass": "kdb_tree.cu"}


def code_only(text: str) -> str:
    """C/C++/CUDA source without its comments and with every run of white
    space collapsed to one blank: what the compiler sees of the code."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":  # a string or character literal, escapes included
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_hash(kind: str) -> str:
    """Hash of the code (comments and layout left out) of the source file
    defining kernel kind `kind` and of every header it includes: a stored ncu
    figure is only reused while that kernel's code is exactly the code it was
    measured on."""
    d = os.path.join(ROOT, "paper_2211_00120_gb300", "csrc")
    h = hashlib.sha256()
    todo, seen = [KIND_SOURCE.get(kind, "")], set()
    while todo:
        f = todo.pop()
        if f in seen or not os.path.isfile(os.path.join(d, f)):
            continue
        seen.add(f)
        with open(os.path.join(d, f), "rb") as fh:
            text = fh.read().decode()
        h.update(f.encode() + code_only(text).encode())
        todo += re.findall(r'#include "([^"/]+)"', text)
    return h.hexdigest()[:16] if seen else ""


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def issue_peak_ginst(device: int = 0):
    """Warp-instruction issue peak of the GPU in G warp-instructions/s: four
    schedulers per SM, one instruction each per cycle, at the maximum SM clock
    of the measured peaks file (the clock the bench's runs hold)."""
    import torch

    sms = torch.cuda.get_device_properties(device).multi_processor_count
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
        src = "4 x SMs x measured max SM clock"
    except Exception:
        mhz, src = 2070.0, "4 x SMs x nominal max SM clock"
    return 4.0 * sms * mhz * 1e6 / 1e9, src


def stored_counters(name: str, kind: str):
    """A committed ncu summary (profiles/<name>.json) if it was taken on the
    current sources of kernel kind `kind`, else None."""
    try:
        with open(os.path.join(ROOT, "profiles", name + ".json")) as f:
            j = json.load(f)
    except Exception:
        return None
    return j if j.get("kernel_hash") == kernel_hash(kind) else None


def kernel_roofline(p: dict, steps: int, points: int, peak_gbs: float, peak_src: str,
                    shapes: dict):
    """Roofline entry of one kernel kind from the library's profiling rows:
    HBM-bound kinds against the copy peak (algorithmic bytes / CUDA-event
    time), the issue-bound local finish against the warp-instruction issue
    peak (instructions from the stored ncu count)."""
    ms = p["ms"]
    if ms <= 0:
        return None
    if p["name"] == "local_finish":
        c = stored_counters("local_finish_instructions", "local_finish")
        peak, src = issue_peak_ginst()
        if c is None:
            return {"kernel": "local_finish", "bound": "alu", "achieved": None, "peak": peak,
                    "unit": "Gwarp-inst/s", "frac": None, "traffic": None, "peak_source": src,
                    "ms_per_step": ms / steps}
        inst = c["warp_instructions_per_point"] * points * steps
        ach = inst / (ms / 1000.0) / 1e9
        return {"kernel": "local_finish", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "Gwarp-inst/s", "frac": ach / peak,
                "traffic": c["dram_bytes_per_point"] * points * p["launches"] / max(p["launches"], 1),
                "warp_instructions_per_point": c["warp_instructions_per_point"],
                "peak_source": src, "ms_per_step": ms / steps,
                "launches_per_step": p["launches"] / steps}
    ach = p["bytes"] / (ms / 1000.0) / 1e9
    traffic = None
    if p["name"] in BYTES_PER_ITEM and p["launches"]:
        items = p["bytes"] / BYTES_PER_ITEM[p["name"]] / p["launches"]
        traffic = traffic_per_launch(p["name"], items, shapes)
    return {"kernel": p["name"], "bound": "hbm", "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
            "frac": ach / peak_gbs, "traffic": traffic, "peak_source": peak_src,
            "ms_per_step": ms / steps, "launches_per_step": p["launches"] / steps,
            "algorithmic_bytes_per_launch": p["bytes"] / max(p["launches"], 1)}


def traffic_per_launch(kind: str, n_items_per_launch: float, shapes: dict):
    """DRAM bytes per launch of `kind` from the committed ncu summary
    (profiles/<kind>_traffic.json, measured on a smaller case and scaled by
    the items a launch processes); None if absent, measured on other kernel
    sources, or with another tile shape than the one in use."""
    p = os.path.join(ROOT, "profiles", f"{kind}_traffic.json")
    try:
        with open(p) as f:
            j = json.load(f)
    except Exception:
        return None
    if not j.get("kernel_hash") or j["kernel_hash"] != kernel_hash(kind):
        return None
    if kind == "radix_pass" and j.get("digit_bits", 8) != shapes.get("digit_bits", 8):
        return None  # counted with another digit width
    shape = shapes.get({"partition_pass": "partition", "radix_pass": "radix"}.get(kind, ""))
    if shape is None:
        return j["dram_bytes_per_item"] * n_items_per_launch
    per_item = j.get("by_shape", {}).get("x".join(str(v) for v in shape))
    return None if per_item is None else per_item * n_items_per_launch


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def floor_bytes(n: int, stride_bytes: int) -> float:
    """Each live record and its one int32 read and written once per level:
    sum over l = 0 .. L-1 of 2 (S + 4) (N - F(l-1))."""
    L = n.bit_length()
    tot = 0.0
    for l in range(L):
        prev = (1 << (l - 1)) - 1 if l >= 1 else 0
        tot += 2.0 * (stride_bytes + 4) * (n - prev)
    return tot


def model_bytes(prof: list, steps: int) -> float:
    """Algorithmic bytes of every launch of one build (the library's profiling
    rows: each kernel's pass model, summed over its launches)."""
    return sum(p["bytes"] for p in prof) / max(steps, 1)


def build_rooflines(prof: list, steps: int, n: int, stride: int, build_ms: float, peak: float,
                    peak_src: str, shapes: dict) -> dict:
    """Roofline entry of the dominant kernel (largest share of the step), each
    big kernel against its own bound, and two whole-build fractions: the
    pass-model bytes of every launch, and the floor bytes (each live record
    and its int32 read and written once per level), each over the peak and
    the build time."""
    dom = max(prof, key=lambda p: p["ms"])
    roof = kernel_roofline(dom, steps, n, peak, peak_src, shapes) or {}
    roof["kernel_share_of_step"] = dom["ms"] / steps / build_ms
    mb = model_bytes(prof, steps)
    roof["build_model_bytes"] = mb
    roof["build_model_frac"] = mb / (peak * 1e9) / (build_ms / 1000.0)
    roof["build_floor_bytes"] = floor_bytes(n, stride)
    roof["build_floor_frac"] = floor_bytes(n, stride) / (peak * 1e9) / (build_ms / 1000.0)
    roof["kernels"] = [r for r in (kernel_roofline(p, steps, n, peak, peak_src, shapes)
                                   for p in prof
                                   if p["name"] in ("partition_pass", "radix_pass", "local_finish"))
                       if r]
    return roof


def timed_builds(kdb, work, src, k: int, mode: int, steps: int, stream):
    """`steps` builds of `work`, each after restoring the input by a device
    copy (which also evicts L2 for inputs above its size), timed with CUDA
    events on the launching stream; returns (ms per build, profiling rows,
    library launches)."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    launches0 = kdb.kdb_launch_count()
    kdb.kdb_profile_start()
    for s in range(steps):
        work.copy_(src)
        ev[s][0].record(stream)
        kdb.kdb_build(work, k, mode)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    prof = kdb.kdb_profile_stop()
    launches = kdb.kdb_launch_count() - launches0
    return [a.elapsed_time(b) for a, b in ev], prof, launches


def tuning_record(kdb, n: int, k: int, stride: int, mode_arg: int):
    """The setting a build of this kind takes (its tuning-table entry, else
    the process-wide setting): a record for the JSON line, and the shapes and
    digit width that select stored counters."""
    (p, r, bits), from_table = kdb.kdb_lookup_tuning(n, k, stride, mode_arg)
    shapes = {"partition": kdb.kdb_tuning_shapes(kdb.TUNE_PARTITION)[p],
              "radix": kdb.kdb_tuning_shapes(kdb.TUNE_RADIX)[r], "digit_bits": bits}
    rec = {"indices": [p, r], "digit_bits": bits, "from_table": from_table,
           "partition_shape": list(shapes["partition"]), "radix_shape": list(shapes["radix"]),
           "shape_fields": ["threads", "items_per_thread", "blocks_per_sm"]}
    return rec, shapes


def workload_leg(kdb, name: str, steps: int, warmup: int, peak: float, peak_src: str) -> dict:
    """One more workload of the build, timed like the headline: device-resident
    input restored before each step, CUDA events, per-kernel rooflines."""
    import torch

    desc, n, k, sf, mode, gen = WORKLOADS[name]
    host = gen(n)
    src = torch.from_numpy(host).cuda()
    work = torch.empty_like(src)
    del host
    stream = torch.cuda.current_stream()
    tuned, shapes = tuning_record(kdb, n, k, 4 * sf, kdb._mode(src, mode))
    for _ in range(warmup):
        work.copy_(src)
        kdb.kdb_build(work, k, mode)
    torch.cuda.synchronize()
    bad = kdb.kdb_validate(work, k, mode)
    if bad != -1:
        raise SystemExit(f"bench: {name}: built array is not a k-d tree (node {bad})")
    times, prof, launches = timed_builds(kdb, work, src, k, mode, steps, stream)
    ms = sum(times) / len(times)
    stride = 4 * sf
    out = {"workload": desc, "n_points": n, "k": k, "stride_bytes": stride,
           "split": ["round_robin", "widest_extent", "widest_tight_box"][mode],
           "steps": steps, "warmup": warmup, "ms_per_step": ms,
           "ms_per_step_median": sorted(times)[len(times) // 2],
           "value": n / (ms / 1000.0) / 1e6, "unit": "Mpts/s", "gpu_launches": launches,
           "kernel_ms_per_step": {p["name"]: round(p["ms"] / steps, 3) for p in prof},
           "tuning": tuned,
           "roofline": build_rooflines(prof, steps, n, stride, ms, peak, peak_src, shapes)}
    del src, work
    torch.cuda.empty_cache()
    return out


def lean_leg(kdb, name: str, steps: int, warmup: int) -> dict:
    """The memory-lean build (kdb_set_memory_mode(MEMORY_LEAN)) of a workload,
    timed like the headline, with its device memory per point beside the
    default build's, and whether its tree equals the default build's."""
    import torch

    desc, n, k, sf, mode, gen = WORKLOADS[name]
    src = torch.from_numpy(gen(n)).cuda()
    work = torch.empty_like(src)
    stream = torch.cuda.current_stream()
    work.copy_(src)
    kdb.kdb_build(work, k, mode)
    want = work.clone()
    prev = kdb.kdb_set_memory_mode(kdb.MEMORY_LEAN)
    try:
        for _ in range(warmup):
            work.copy_(src)
            kdb.kdb_build(work, k, mode)
        torch.cuda.synchronize()
        equal = bool(torch.equal(work.view(torch.int32), want.view(torch.int32)))
        times, prof, launches = timed_builds(kdb, work, src, k, mode, steps, stream)
    finally:
        kdb.kdb_set_memory_mode(prev)
    del src, work, want
    torch.cuda.empty_cache()
    ms = sum(times) / len(times)
    stride = 4 * sf
    return {"workload": desc, "memory_mode": "lean", "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "ms_per_step_median": sorted(times)[len(times) // 2],
            "value": n / (ms / 1000.0) / 1e6, "unit": "Mpts/s", "gpu_launches": launches,
            "workspace_bytes_per_point": kdb.kdb_lean_workspace_size(n, k, stride, mode) / n,
            "default_workspace_bytes_per_point": kdb.load().kdb_workspace_size(n, k, stride, mode) / n,
            "equal_to_default_build": equal,
            "kernel_ms_per_step": {p["name"]: round(p["ms"] / steps, 3) for p in prof},
            "timing": "CUDA events around each synchronous kdb_build call (host decisions between "
                      "the top levels' passes included)"}


def host_info() -> dict:
    """CPU model and core counts of the host the CPU baselines run on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model Name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"cpu_model": model, "nproc": len(os.sched_getaffinity(0)),
            "machine": os.uname().machine}


def host_link(t, device: int) -> dict:
    """Where the pinned host records live: the NUMA node of a sample of the
    buffer's pages (move_pages in query mode), the NUMA node the GPU's PCI
    function reports, and the nodes that have CPUs."""
    import ctypes

    info = {"gpu_numa_node": None, "pages_numa_nodes": None, "cpu_numa_nodes": None}
    try:
        import torch

        pr = torch.cuda.get_device_properties(device)
        bus = (f"{getattr(pr, 'pci_domain_id', 0):04x}:{pr.pci_bus_id:02x}:"
               f"{pr.pci_device_id:02x}.0")
        with open(f"/sys/bus/pci/devices/{bus}/numa_node") as f:
            info["gpu_numa_node"] = int(f.read().strip())
        info["gpu_pci"] = bus
    except Exception:
        pass
    try:
        nodes = {}
        base = "/sys/devices/system/node"
        for d in sorted(os.listdir(base)):
            if d.startswith("node") and d[4:].isdigit():
                with open(os.path.join(base, d, "cpulist")) as f:
                    cl = f.read().strip()
                if cl:
                    nodes[int(d[4:])] = cl
        info["cpu_numa_nodes"] = nodes
    except Exception:
        pass
    try:
        nr = {"x86_64": 279, "aarch64": 239}[os.uname().machine]
        libc = ctypes.CDLL(None, use_errno=True)
        page = os.sysconf("SC_PAGE_SIZE")
        nbytes = t.numel() * t.element_size()
        m = 64
        addrs = [(t.data_ptr() + i * (nbytes // m)) & ~(page - 1) for i in range(m)]
        pages = (ctypes.c_void_p * m)(*addrs)
        status = (ctypes.c_int * m)()
        libc.syscall.restype = ctypes.c_long
        rc = libc.syscall(ctypes.c_long(nr), ctypes.c_int(0), ctypes.c_ulong(m), pages, None,
                          status, ctypes.c_int(0))
        if rc == 0:
            hist = {}
            for v in status:
                hist[str(v)] = hist.get(str(v), 0) + 1
            info["pages_numa_nodes"] = hist
    except Exception:
        pass
    return info


def cpu_baseline(workload: str, target_s: float = 15.0):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload: the first n points of the same generator, n grown until one
    build takes a few seconds, then repeated to about target_s seconds."""
    from oracle import oracle

    desc, n_full, k, sf, mode, gen = WORKLOADS[workload]
    n = 1 << 18
    pts = gen(n_full if n_full <= (1 << 22) else (1 << 22))
    while True:
        sample = np.ascontiguousarray(pts[:n])
        t0 = time.perf_counter()
        oracle.build(sample, k, mode)
        dt = time.perf_counter() - t0
        if dt > target_s / 4 or n >= pts.shape[0]:
            break
        n *= 2
    reps, total = 1, dt
    while total < target_s:
        t0 = time.perf_counter()
        oracle.build(sample, k, mode)
        total += time.perf_counter() - t0
        reps += 1
    return {"value": reps * n / total / 1e6, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} builds of the first {n} points of the same generator "
                      f"({desc}); oracle single-threaded, {total:.1f} s", **host_info()}


def cpu_parallel_baseline(workload: str, log2_points: int = 24):
    """The paper's level loop ported to host threads (oracle/paper_cpu.c, one
    thread per core) on a bounded sample: the first 2^log2_points points of
    the workload's generator."""
    from oracle import paper_cpu

    desc, n_full, k, sf, mode, gen = WORKLOADS[workload]
    n = min(n_full, 1 << log2_points)
    pts = gen(n)
    paper_cpu.build(pts[:4096], k, mode)  # load the library
    t0 = time.perf_counter()
    paper_cpu.build(pts, k, mode)
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e6, "unit": "Mpts/s", "cores": paper_cpu.cores(),
            "kind": "paper level loop on host threads (parallel sort per level + tag update)",
            "sample": f"one build of the first {n} points of the same generator ({desc}), "
                      f"{dt:.1f} s", **host_info()}


def batched_vs_serial(sets: int = 4096, lo: int = 100, hi: int = 1_000_000, seed: int = 3,
                      steps: int = 3, world: int = 1, rank: int = 0, dist=None):
    """Many independent float3 sets (sizes log-uniform in [lo, hi], uniform
    points, round robin) built by one kdb_build_batched call against one
    kdb_build call per set, on the same device-resident array: builds/s of
    each, and whether the outputs are identical.  With several ranks every
    rank takes its LPT share of the sets (no exchange); times are the max
    over ranks."""
    import torch
    from paper_2211_00120_gb300 import kdb, shard
    sizes_all = synth.lognormal_sizes(sets, lo, hi, seed=seed)
    offs_all = np.concatenate([[0], np.cumsum(sizes_all)]).astype(np.int64)
    n_all = int(offs_all[-1])
    mine = shard.lpt_shards([int(v) for v in sizes_all], world)[rank]
    sizes = sizes_all[mine]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rows = [synth.uniform_rows(int(offs_all[b]), int(sizes_all[b]), 3, seed=seed) for b in mine]
    host = np.concatenate(rows) if rows else np.zeros((0, 3), np.float32)
    src = torch.from_numpy(host).cuda()
    work = torch.empty_like(src)
    stream = torch.cuda.current_stream()
    off_list = offs.tolist()
    nsets = len(mine)

    def batched():
        kdb.kdb_build_batched(work, off_list, 3, kdb.ROUND_ROBIN)

    def serial():
        for b in range(nsets):
            if off_list[b + 1] > off_list[b]:
                kdb.kdb_build(work[off_list[b]:off_list[b + 1]], 3, kdb.ROUND_ROBIN)

    def timed(fn):
        times = []
        for _ in range(steps):
            work.copy_(src)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return statistics.median(times)

    work.copy_(src)
    batched()  # warm-up (pool, first launches)
    out_b = work.clone()
    work.copy_(src)
    serial()
    equal = bool(torch.equal(work.view(torch.int32), out_b.view(torch.int32)))
    tb = timed(batched)
    ts = timed(serial)
    # the same batched build from a plan captured into one CUDA graph
    plan = kdb.Plan(off_list, 3, 12, kdb.ROUND_ROBIN)
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            plan.enqueue(work, stream=cap)
    stream.wait_stream(cap)
    work.copy_(src)
    graph.replay()
    plan.status()
    equal = equal and bool(torch.equal(work.view(torch.int32), out_b.view(torch.int32)))
    tg = timed(graph.replay)
    del graph
    plan.close()
    del src, work, out_b
    torch.cuda.empty_cache()
    if dist is not None:
        t = torch.tensor([tb, ts, tg, 0.0 if equal else 1.0], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tb, ts, tg, equal = float(t[0]), float(t[1]), float(t[2]), float(t[3]) == 0.0
    n = n_all
    return {"workload": f"{sets} float3 sets, sizes log-uniform in [{lo}, {hi}] (seed {seed}), "
                        f"{n} points uniform in [0,1)^3, round robin",
            "ranks": world, "sharding": "LPT by points x levels, no exchange" if world > 1 else None,
            "points": n, "batched_ms": tb, "serial_ms": ts, "graph_ms": tg,
            "graph_builds_per_s": sets / (tg / 1000.0),
            "batched_builds_per_s": sets / (tb / 1000.0), "serial_builds_per_s": sets / (ts / 1000.0),
            "batched_mpts_per_s": n / (tb / 1000.0) / 1e6, "speedup": ts / tb,
            "equal_output": equal, "steps": steps,
            "timing": "CUDA events around the whole call (serial: 4096 synchronous kdb_build calls)"}


def serving(rate: float = 2000.0, duration_s: float = 5.0, lo: int = 1000, hi: int = 10_000_000,
            budget_gb: float = 40.0, seed: int = 4, inflight: int = 3, pool_log: int = 24):
    """The build server under a Poisson stream of requests: sizes log-uniform
    in [lo, hi], float3 or float4 records, uniform or clustered points (fair
    coins), every request copied in from pinned host memory and its tree
    copied back out.  The payloads are slices of four pre-generated pinned
    pools, so host generation is not timed.  Reports builds/s and latency
    percentiles (submit to copy-back done) at the offered rate; if that rate
    saturates the server, again at 80% of the throughput it reached; and the
    same requests served one at a time (one stream, one request per batch)."""
    import torch
    from paper_2211_00120_gb300 import kdb

    P = 1 << pool_log
    pools = {}
    for f4 in (False, True):
        for cl in (False, True):
            base = synth.mixed(P, 3, seed=60 + cl) if cl else synth.uniform(P, 3, seed=60)
            if f4:
                arr = np.empty((P, 4), dtype=np.float32)
                arr[:, :3] = base
                arr[:, 3] = np.arange(P, dtype=np.uint32).view(np.float32)
            else:
                arr = base
            pools[(f4, cl)] = (torch.from_numpy(arr).pin_memory(),
                               torch.empty(arr.shape, dtype=torch.float32).pin_memory())
    t_arr, sizes, f4s, cls, where = synth.poisson_requests(rate, duration_s, lo, hi, seed=seed)
    sizes = np.minimum(sizes, P)
    reqs = []
    for i in range(len(t_arr)):
        n = int(sizes[i])
        off = int(where[i] * (P - n + 1))
        src, dst = pools[(bool(f4s[i]), bool(cls[i]))]
        reqs.append((float(t_arr[i]), src[off:off + n], dst[off:off + n]))

    def run(scale: float, count: int, **cfg):
        """Replays the first `count` requests with arrival times / scale."""
        srv = kdb.Server(budget_bytes=int(budget_gb * (1 << 30)), **cfg)
        done, late = {}, 0.0
        t0 = time.perf_counter()
        for t, src, dst in reqs[:count]:
            target = t0 + t / scale
            while True:
                d = target - time.perf_counter()
                if d <= 0:
                    break
                if d > 0.0006:
                    time.sleep(d - 0.0004)
            late = max(late, time.perf_counter() - target)
            srv.submit(src, 3, kdb.ROUND_ROBIN, out=dst)
            for r in srv.poll(0):
                done[r["id"]] = r
        while len(done) < count:
            for r in srv.poll(200):
                done[r["id"]] = r
        st = srv.stats()
        srv.close()
        rs = list(done.values())
        bad = sum(1 for r in rs if r["status"] != kdb.OK)
        first = min(r["submit_s"] for r in rs)
        last = max(r["done_s"] for r in rs)
        lat = np.array([r["done_s"] - r["submit_s"] for r in rs]) * 1e3
        pts = sum(r["n"] for r in rs)
        offered = count / (reqs[count - 1][0] / scale) if count > 1 else None
        achieved = count / (last - first)
        return {"offered_builds_per_s": offered, "builds_per_s": achieved,
                "mpts_per_s": pts / (last - first) / 1e6, "requests": count, "failed": bad,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "saturated": bool(offered and achieved < 0.95 * offered),
                "batches": st["batches"], "max_batch_requests": st["max_batch_requests"],
                "max_inflight_batches": st["max_inflight_batches"],
                "max_used_gb": st["max_used_bytes"] / 2**30, "max_submit_lateness_ms": late * 1e3}

    nreq = len(reqs)
    out = {"workload": f"Poisson arrivals at {rate:g} req/s for {duration_s:g} s ({nreq} requests, "
                       f"seed {seed}), sizes log-uniform in [{lo}, {hi}], float3/float4 and "
                       f"uniform/clustered 50/50, round robin, {budget_gb:g} GB budget",
           "latency": "submit to the end of the copy back to pinned host memory (server clock)",
           "inflight_batches": inflight}
    out["offered"] = run(1.0, nreq, max_inflight_batches=inflight)
    if out["offered"]["saturated"]:
        scale = 0.8 * out["offered"]["builds_per_s"] / rate
        out["at_80pct_of_max"] = run(scale, nreq, max_inflight_batches=inflight)
    # the same stream served one request at a time: 2 s of arrivals
    m = int(np.searchsorted(t_arr, 2.0))
    one = run(1.0, m, max_inflight_batches=1, max_batch_requests=1)
    cb = run(1.0, m, max_inflight_batches=inflight)
    out["one_at_a_time_vs_batched"] = {"requests": m, "one_at_a_time_builds_per_s": one["builds_per_s"],
                                       "batched_builds_per_s": cb["builds_per_s"],
                                       "one_at_a_time_p50_ms": one["p50_ms"],
                                       "batched_p50_ms": cb["p50_ms"],
                                       "speedup": cb["builds_per_s"] / one["builds_per_s"]}
    del pools, reqs
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    desc, n_full, k, sf, mode, gen = WORKLOADS[args.workload]
    # each step: one oracle build of a bounded sample, so the run stays short
    n = 1 << 20
    pts = np.ascontiguousarray(gen(n_full)[:n]) if n_full <= n else gen(n)
    from oracle import oracle

    for _ in range(args.warmup):
        oracle.build(pts, k, mode)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.build(pts, k, mode)
        t.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(t) / len(t)
    val = n / (ms / 1000.0) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": desc, "sample_points": n, "k": k,
                                            "stride_bytes": 4 * sf},
            "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {n} points of the workload per step",
                             **host_info()},
            "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uniform_1e8_f3_rr", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched vs serial measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the 1e7 mixed and 1e8 float4 widest-extent workloads")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving measurement (prints its JSON object)")
    ap.add_argument("--points", type=int, default=0,
                    help="override the workload's number of points (small profiling cases)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tile shapes instead of timing the compiled ones first")
    ap.add_argument("--tuning", default="",
                    help="partition,radix tile-shape indices[,digit bits] to use (skips the autotuner)")
    ap.add_argument("--profile-only", action="store_true",
                    help="warm-up and one build, nothing timed (for ncu launch lists)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.profile_only:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2211_00120_gb300 import kdb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.serving_only:
        print(json.dumps(serving()), flush=True)
        return 0
    desc, n, k, sf, mode, gen = WORKLOADS[args.workload]
    if args.points:
        n = args.points
        desc = f"{desc} [first {n} points]"
    host = gen(n)
    stride = 4 * sf
    src = torch.from_numpy(host).cuda()
    work = torch.empty_like(src)
    stream = torch.cuda.current_stream()

    # tile shapes of the two sort kernels: timed on this workload before the
    # warm-up (kdb_autotune builds a copy of the points), or given
    autotune = None
    if args.tuning:
        kdb.kdb_set_tuning(*(int(v) for v in args.tuning.split(",")))
    elif not args.no_autotune and not args.profile_only:
        r = kdb.kdb_autotune(src, k, mode, reps=3)
        autotune = {"best": list(r["best"]), "best_ms": r["best_ms"],
                    "ms": {f"{p},{q},{b}": round(v, 3) for (p, q, b), v in sorted(r["ms"].items())},
                    "key_fields": ["partition_shape", "radix_shape", "digit_bits"]}
    tuned, shapes = tuning_record(kdb, n, k, stride, kdb._mode(src, mode))
    tuned["autotune"] = autotune

    for _ in range(args.warmup):
        work.copy_(src)
        kdb.kdb_build(work, k, mode)
    torch.cuda.synchronize()
    if args.profile_only:
        work.copy_(src)
        kdb.kdb_build(work, k, mode)
        torch.cuda.synchronize()
        return 0
    bad = kdb.kdb_validate(work, k, mode)
    if bad != -1:
        raise SystemExit(f"bench: built array is not a k-d tree (node {bad})")

    sampler = ClockSampler(local)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    step_ms, prof, launches = timed_builds(kdb, work, src, k, mode, args.steps, stream)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = sorted(step_ms)
    ms = sum(step_ms) / args.steps
    ms_median = step_ms[len(step_ms) // 2]
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n / (ms / 1000.0) / 1e6

    # roofline of the dominant kernel (largest share of the step), each kernel
    # against its own bound: the sort passes against the HBM copy peak
    # (algorithmic bytes over their CUDA-event time in the timed steps), the
    # issue-bound local finish against the warp-instruction issue peak
    peak, peak_src = measured_peak()
    kernel_ms = {p["name"]: round(p["ms"] / args.steps, 3) for p in prof}
    roofline = build_rooflines(prof, args.steps, n, stride, ms, peak, peak_src, shapes)

    # the paper's almost-in-place placement (one int32 per point) on the same
    # builds, for comparison with the default gather through spare workspace
    prev = kdb.kdb_set_placement(kdb.PLACEMENT_IN_PLACE)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(3)]
    kdb.kdb_profile_start()
    for e0, e1 in ev2:
        work.copy_(src)
        e0.record(stream)
        kdb.kdb_build(work, k, mode)
        e1.record(stream)
    torch.cuda.synchronize()
    prof_ip = {p["name"]: p["ms"] / len(ev2) for p in kdb.kdb_profile_stop()}
    kdb.kdb_set_placement(prev)
    in_place = {"ms_per_step": sum(a.elapsed_time(b) for a, b in ev2) / len(ev2),
                "placement_ms": round(prof_ip.get("placement", 0.0), 3), "steps": len(ev2)}

    e2e = None
    if not args.no_e2e:
        h_src = torch.from_numpy(host)
        h = torch.empty_like(h_src).pin_memory()
        times = []
        # untimed calls first (as many as the device legs' warm-up): the
        # device's first accesses to freshly pinned pages over the host link
        # are slow, as any first use is
        e_warm = max(3, args.warmup)
        for s in range(e_warm + max(1, args.e2e_steps)):
            h.copy_(h_src)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kdb.kdb_build_host(h, k, mode)
            if s >= e_warm:
                times.append(time.perf_counter() - t0)
        e_ms = 1000.0 * sum(times) / len(times)
        # one more call, not timed, with the library's per-kernel events: which
        # kernels the host link slows down (those that touch host records)
        h.copy_(h_src)
        torch.cuda.synchronize()
        kdb.kdb_profile_start()
        kdb.kdb_build_host(h, k, mode)
        e_kernel_ms = {p["name"]: round(p["ms"], 3) for p in kdb.kdb_profile_stop()}
        mapped = stride == 4 * k and k <= 3
        link = host_link(h, local)
        pre = e_kernel_ms.get("prepass")
        if mapped and pre:
            # the prepass reads every host record once over the host link
            link["prepass_ms"] = pre
            link["prepass_read_gbs"] = n * stride / (pre / 1000.0) / 1e9
        e2e = {"value": world * n / (e_ms / 1000.0) / 1e6, "unit": "Mpts/s",
               "host_link": link,
               "h2d_bytes_per_step": n * stride, "d2h_bytes_per_step": n * stride,
               "ms_per_step": e_ms, "steps": len(times), "warmup": e_warm,
               "kernel_ms_one_call": e_kernel_ms,
               "api": "kdb_build_host on a pinned host tensor",
               "transfer": ("the kernels read the host records and write the tree into them "
                            "over the host link, no device copy of the records")
               if mapped else "chunked copies to the device overlapped with the first pass, "
                              "one copy back"}

    legs = {}
    if not args.no_legs and not args.points:
        del src, work
        torch.cuda.empty_cache()
        src = work = None
        for name in ("mixed_1e7_f3_rr", "aniso_1e8_f4_widest"):
            if name != args.workload:
                legs[name] = workload_leg(kdb, name, min(args.steps, 20), args.warmup, peak, peak_src)
        legs["lean_" + args.workload] = lean_leg(kdb, args.workload, min(args.steps, 5), args.warmup)

    batched = None
    if not args.no_batched:
        del src, work
        torch.cuda.empty_cache()
        batched = batched_vs_serial(world=world, rank=rank, dist=dist)

    served = None
    if world == 1 and not args.no_serving:
        served = serving()

    cpu = cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
        cpu_par = cpu_parallel_baseline(args.workload)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "ms_per_step_median": ms_median,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": desc, "n_points": n, "k": k, "stride_bytes": stride,
                           "split": ["round_robin", "widest_extent", "widest_tight_box"][mode],
                           "parallelism": "replicas" if world > 1 else "single_gpu",
                           "l2": "input 1.2+ GB > L2, restored by a device copy before each step"},
                "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_parallel": cpu_par,
                "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "kernel_ms_per_step": kernel_ms,
                "placement_in_place": in_place, "tuning": tuned, "workloads": legs,
                "batched": batched,
                "serving": served}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
