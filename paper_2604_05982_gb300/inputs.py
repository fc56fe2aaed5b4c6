"""Seeded synthetic inputs shared by the GPU path, the oracle tests and the bench.

This module holds input generation only: none of the fork-join method's
arithmetic lives here.  Every stream is the SplitMix64 generator (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) used
as a counter-based source: the k-th output (k = 0, 1, ...) of the stream seeded
``s`` is ``mix64(s + (k + 1) * 0x9E3779B97F4A7C15)``, so any slice of a stream
can be produced in one vectorised numpy pass.

Recipes (the workload shapes of the paper's evaluation, Sec. 6):

* ``keys_u32(n, seed=1)``: low 32 bits of successive outputs -> uniform uint32
  keys for the mergesort workload (Cilksort, Sec. 6.3.1).
* ``rmat_graph(scale, ef=16, a, b, c, seed)``: R-MAT edge sampling, the
  synthetic stand-in for the SNAP graphs of the k-clique study (Sec. 6.4.2),
  which are not available here.  ``ef * 2**scale`` directed samples; for sample
  ``e`` and level ``l`` (``0 <= l < scale``, most significant bit first) draw
  ``u = (out[e*scale+l] >> 11) * 2**-53`` and pick quadrant (0,0) if ``u < a``,
  (0,1) if ``u < a+b``, (1,0) if ``u < a+b+c``, else (1,1).  No noise and no
  vertex permutation.  Edges are then made undirected as (min, max), self
  loops dropped and duplicates removed.  Isolated vertices are kept.
* ``fmm_points(n, dist, seed=3)``: particle positions and charges for the
  Laplace FMM (Sec. 6.4.1).  ``uniform``: 3 draws per point from stream
  ``seed`` -> unit cube.  ``plummer``: radius from stream ``seed ^ R_SALT``
  by inversion of the Plummer cumulative mass with scale a = 1,
  ``r = 1/sqrt(U**(-2/3) - 1)``, rejecting r > 10 (the accepted values in
  stream order); direction uniform on the sphere from stream ``seed ^ D_SALT``
  (``cos(theta) = 2U - 1``, ``phi = 2 pi U``).  Charges U(-1, 1) from stream
  ``seed ^ Q_SALT``.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

R_SALT = 0x5243_0000_0000_0001  # radius sub-stream of the Plummer recipe
D_SALT = 0x4449_0000_0000_0002  # direction sub-stream
Q_SALT = 0x5143_0000_0000_0003  # charge sub-stream


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64_stream(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream seeded ``seed``."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN
    return _mix64(state)


def u01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    return (splitmix64_stream(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def keys_u32(n: int, seed: int = 1) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        out[s:s + c] = (splitmix64_stream(seed, s, c) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, seed: int = 7):
    """Undirected simple R-MAT graph: returns (n_vertices, edges[m, 2] int32 with u < v, sorted)."""
    n = 1 << scale
    n_samples = edge_factor * n
    t1, t2, t3 = a, a + b, a + b + c
    src = np.zeros(n_samples, dtype=np.int64)
    dst = np.zeros(n_samples, dtype=np.int64)
    idx = np.arange(n_samples, dtype=np.int64) * scale
    for level in range(scale):
        # draw index e*scale + level, taken in chunks to bound memory
        u = np.empty(n_samples, dtype=np.float64)
        chunk = 1 << 23
        for s in range(0, n_samples, chunk):
            cidx = idx[s:s + chunk] + level
            k = cidx.astype(np.uint64) + np.uint64(1)
            with np.errstate(over="ignore"):
                state = np.uint64(seed) + k * GOLDEN
            u[s:s + chunk] = (_mix64(state) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        bit = np.int64(1) << np.int64(scale - 1 - level)
        sbit = u >= t2                      # quadrants (1,0) and (1,1)
        dbit = ((u >= t1) & (u < t2)) | (u >= t3)   # quadrants (0,1) and (1,1)
        src += sbit.astype(np.int64) * bit
        dst += dbit.astype(np.int64) * bit
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    keep = lo != hi
    key = np.unique(lo[keep] * n + hi[keep])
    edges = np.stack([key // n, key % n], axis=1).astype(np.int32)
    return n, edges


def random_graph(n: int, p: float, seed: int):
    """Erdos-Renyi G(n, p) for small test graphs: edges (u < v) sorted, int32."""
    iu, ju = np.triu_indices(n, k=1)
    u = u01(seed, 0, len(iu))
    keep = u < p
    return n, np.stack([iu[keep], ju[keep]], axis=1).astype(np.int32)


def fmm_points(n: int, dist: str = "uniform", seed: int = 3):
    """Positions (n, 3) float64 and charges (n,) float64."""
    if dist == "uniform":
        pos = u01(seed, 0, 3 * n).reshape(n, 3)
    elif dist == "plummer":
        radii = np.empty(0, dtype=np.float64)
        start = 0
        while radii.size < n:
            want = int((n - radii.size) * 1.01) + 1024
            U = u01(seed ^ R_SALT, start, want)
            start += want
            with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
                r = 1.0 / np.sqrt(U ** (-2.0 / 3.0) - 1.0)
            ok = np.isfinite(r) & (r <= 10.0)
            radii = np.concatenate([radii, r[ok]])
        r = radii[:n]
        d = u01(seed ^ D_SALT, 0, 2 * n).reshape(n, 2)
        ct = 2.0 * d[:, 0] - 1.0
        st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
        ph = 2.0 * np.pi * d[:, 1]
        pos = np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * ct], axis=1)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    q = 2.0 * u01(seed ^ Q_SALT, 0, n) - 1.0
    return np.ascontiguousarray(pos), q


def poisson_trace(n_requests: int, rate_per_s: float, seed: int):
    """Arrival times (seconds, increasing) of a Poisson process, and a per-request uniform draw."""
    u = u01(seed, 0, 2 * n_requests).reshape(n_requests, 2)
    gaps = -np.log1p(-u[:, 0]) / rate_per_s
    return np.cumsum(gaps), u[:, 1]
