"""Seeded synthetic point sets.

This module only draws random numbers; it holds no part of the k-d tree build.
Tests (which feed the CPU oracle) and the benchmark (which feeds the CUDA
library) both take their inputs from here, so both sides see identical bytes.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) in counter form: draw i of a stream is
``mix64(key + (i + 1) * GOLDEN)``, with ``mix64`` the SplitMix64 finaliser.
A stream's key is ``mix64(seed) ^ mix64(stream_id + GOLDEN)``.

Workload shapes follow the paper's experiments (uniform random points,
Sec. 7.1, Table 1) and the configurations the library is measured on:

* ``uniform``: i.i.d. uniform in [0,1)^k; u = (x >> 40) * 2^-24 is exact in
  float32.
* ``mixed``: half uniform, half drawn from 64 isotropic Gaussian clusters
  (sigma 0.01, centres uniform in [0,1)^k, Box-Muller in float64, cast to
  float32, no clamping), then 1% of the rows overwritten by exact copies of
  other random rows, then shuffled by sorting random 64-bit keys.
* ``aniso_float4``: x in U[0,100), y in U[0,1), z in U[0,10), and a fourth
  float that carries the uint32 bit pattern of the row index (payload).
* ``lognormal_sizes``: set sizes floor(exp(U[ln lo, ln hi])).
* ``int32_uniform``: int32 coordinates uniform over the whole range (the
  paper's int1 data, Table 1).
* ``poisson_requests``: a Poisson stream of build requests for the serving
  measurement: exponential gaps, log-uniform sizes, float3/float4 and
  uniform/clustered by fair coins.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream_id: int) -> np.uint64:
    a = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        b = _mix64(np.array([stream_id & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) + GOLDEN)[0]
    return np.uint64(a ^ b)


def u64(seed: int, stream_id: int, n: int, start: int = 0) -> np.ndarray:
    """Draws [start, start+n) of stream (seed, stream_id) as uint64."""
    key = stream_key(seed, stream_id)
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64) * GOLDEN + key
    return _mix64(ctr)


def unit_f32(x: np.ndarray) -> np.ndarray:
    """uint64 -> float32 uniform in [0,1), exactly representable."""
    return ((x >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)).astype(np.float32)


def unit_f64(x: np.ndarray) -> np.ndarray:
    """uint64 -> float64 uniform in [0,1)."""
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(n: int, k: int = 3, seed: int = 0, stream: int = 0) -> np.ndarray:
    """(n, k) float32, i.i.d. uniform in [0,1)^k."""
    out = np.empty((n, k), dtype=np.float32)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        out[s:s + m] = unit_f32(u64(seed, stream, m * k, s * k)).reshape(m, k)
    return out


def uniform_rows(start: int, n: int, k: int = 3, seed: int = 0, stream: int = 0) -> np.ndarray:
    """Rows [start, start + n) of uniform(., k, seed, stream), drawn alone."""
    return unit_f32(u64(seed, stream, n * k, start * k)).reshape(n, k)


def _gauss(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals (float64) by Box-Muller."""
    a = u64(seed, stream, n)
    b = u64(seed, stream + 1, n)
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u2 = unit_f64(b)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def permutation(n: int, seed: int, stream: int) -> np.ndarray:
    """A seeded permutation of range(n): argsort of random 64-bit keys."""
    return np.argsort(u64(seed, stream, n), kind="stable")


def mixed(n: int, k: int = 3, seed: int = 1, clusters: int = 64, sigma: float = 0.01,
          dup_frac: float = 0.01) -> np.ndarray:
    """Half uniform, half Gaussian clusters, 1% exact duplicates, shuffled."""
    n_uni = n // 2
    n_cl = n - n_uni
    pts = np.empty((n, k), dtype=np.float32)
    pts[:n_uni] = uniform(n_uni, k, seed, stream=10)
    centres = unit_f64(u64(seed, 11, clusters * k)).reshape(clusters, k)
    which = (u64(seed, 12, n_cl) % np.uint64(clusters)).astype(np.int64)
    g = _gauss(seed, 13, n_cl * k).reshape(n_cl, k)
    pts[n_uni:] = (centres[which] + sigma * g).astype(np.float32)
    n_dup = int(n * dup_frac)
    if n_dup > 0:
        dst = permutation(n, seed, 15)[:n_dup]
        src = (u64(seed, 16, n_dup) % np.uint64(n)).astype(np.int64)
        pts[dst] = pts.copy()[src]
    return np.ascontiguousarray(pts[permutation(n, seed, 17)])


def aniso_float4(n: int, seed: int = 2, box=(100.0, 1.0, 10.0)) -> np.ndarray:
    """(n, 4) float32: xyz uniform in the box, w = bits of uint32 row index."""
    out = np.empty((n, 4), dtype=np.float32)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        u = unit_f64(u64(seed, 20, 3 * m, 3 * s)).reshape(m, 3)
        for d in range(3):
            out[s:s + m, d] = (u[:, d] * box[d]).astype(np.float32)
    out[:, 3] = np.arange(n, dtype=np.uint32).view(np.float32)
    return out


def lognormal_sizes(count: int, lo: float, hi: float, seed: int = 3) -> np.ndarray:
    """count set sizes floor(exp(U[ln lo, ln hi])) (log-uniform)."""
    u = unit_f64(u64(seed, 30, count))
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def with_stride(points: np.ndarray, stride_floats: int, payload_seed: int = 99) -> np.ndarray:
    """Pads records to ``stride_floats`` 4-byte words with seeded payload bits."""
    n, k = points.shape
    if stride_floats < k:
        raise ValueError("stride smaller than k")
    out = np.empty((n, stride_floats), dtype=np.float32)
    out[:, :k] = points
    if stride_floats > k:
        # arbitrary bit patterns, NaNs included: payload is moved, never compared
        bits = (u64(payload_seed, 40, n * (stride_floats - k)) >> np.uint64(32)).astype(np.uint32)
        out[:, k:] = bits.reshape(n, stride_floats - k).view(np.float32)
    return out


def poisson_requests(rate: float, duration_s: float, lo: float, hi: float, seed: int = 4):
    """A Poisson stream of build requests: arrival times (seconds, exponential
    gaps of mean 1/rate, up to duration_s), sizes log-uniform in [lo, hi], and
    per request two fair coins: float4 records (else float3) and clustered
    points (else uniform)."""
    m = int(rate * duration_s * 1.2 + 64)
    gaps = -np.log(1.0 - unit_f64(u64(seed, 50, m))) / rate
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    c = len(t)
    u = unit_f64(u64(seed, 51, c))
    sizes = np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    coins = u64(seed, 52, c)
    float4 = (coins & np.uint64(1)).astype(bool)
    clustered = ((coins >> np.uint64(1)) & np.uint64(1)).astype(bool)
    where = unit_f64(u64(seed, 53, c))  # position of the request's points in a pool
    return t, sizes, float4, clustered, where


def int32_uniform(n: int, k: int = 1, seed: int = 0, stream: int = 60) -> np.ndarray:
    """(n, k) int32, i.i.d. uniform over the whole int32 range (the top 32 bits
    of each SplitMix64 draw)."""
    out = np.empty((n, k), dtype=np.int32)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        out[s:s + m] = (u64(seed, stream, m * k, s * k) >> np.uint64(32)).astype(np.uint32).view(
            np.int32).reshape(m, k)
    return out
