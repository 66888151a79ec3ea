"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's callers.

This module draws random graphs and random adjoints.  It holds none of the
shortest-path arithmetic: it never relaxes an edge, never compares a path and
never imports the oracle or the CUDA library.  Both sides of every parity test
receive their inputs from here.

Every random number is a pure function of (seed, position) through SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; the finaliser constants are the published ones).  The same counter
scheme is implemented on the device in ``graphgen_dev.cu``; the two are checked
to be bit-identical by the tests.

Counter layout for element (i, j) of an n-vertex graph and stream s in {0, 1}:

    h(seed, i, j, s) = splitmix64(seed * GAMMA + (((i * n + j) << 1) | s))   (mod 2**64)

* edge (i, j) present  iff  (h(.., 1) >> 11) * 2**-53 < p
* int32 weight         =  lo + h(.., 0) mod (hi - lo + 1)
* fp32 weight in (0,1] =  ((h(.., 0) >> 40) + 1) * 2**-24
* fp32 weight in [1,2) =  1 + (h(.., 0) >> 40) * 2**-24
* fp64 weight in (0,1] =  ((h(.., 0) >> 11) + 1) * 2**-53
* fp64 weight in [1,2) =  1 + (h(.., 0) >> 12) * 2**-52
* int64 weight         =  lo + h(.., 0) mod (hi - lo + 1)
* D[i][i] = 0; a missing edge is INF (2**29 for int32, 2**61 for int64, +inf
  for the floating types).

The paper's own inputs are synthetic dense distance matrices with a share of
null entries (Sec. 4.1); no public dataset is involved.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
INF_I32 = 1 << 29
INF_I64 = 1 << 61

KIND_UNIT = 0      # fp32 weights in (0, 1]
KIND_ONE_TWO = 1   # fp32 weights in [1, 2)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 counters."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _counters(seed: int, n: int, rows: np.ndarray, s: int) -> np.ndarray:
    i = rows.astype(np.uint64)[:, None]
    j = np.arange(n, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        base = np.uint64(seed) * GAMMA
        lin = (i * np.uint64(n) + j) << np.uint64(1)
        return base + (lin | np.uint64(s))


def _edge_mask(seed: int, n: int, rows: np.ndarray, p: float) -> np.ndarray:
    h1 = splitmix64(_counters(seed, n, rows, 1))
    u = (h1 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return u < p


def dense_graph_i32(n: int, seed: int, p: float, lo: int, hi: int,
                    inf: int = INF_I32, rows=None, chunk_rows: int = 1024) -> np.ndarray:
    """Directed graph with int32 weights uniform in [lo, hi]; returns rows x n."""
    rows = np.arange(n) if rows is None else np.asarray(rows)
    out = np.empty((len(rows), n), dtype=np.int32)
    span = np.uint64(hi - lo + 1)
    for s in range(0, len(rows), chunk_rows):
        rr = rows[s:s + chunk_rows]
        h0 = splitmix64(_counters(seed, n, rr, 0))
        w = (np.int64(lo) + (h0 % span).astype(np.int64)).astype(np.int32)
        m = _edge_mask(seed, n, rr, p)
        blk = np.where(m, w, np.int32(inf))
        blk[np.arange(len(rr)), rr] = 0
        out[s:s + chunk_rows] = blk
    return out


def dense_graph_f32(n: int, seed: int, p: float, kind: int = KIND_UNIT,
                    rows=None, chunk_rows: int = 1024) -> np.ndarray:
    """Directed graph with fp32 weights in (0,1] (KIND_UNIT) or [1,2) (KIND_ONE_TWO)."""
    rows = np.arange(n) if rows is None else np.asarray(rows)
    out = np.empty((len(rows), n), dtype=np.float32)
    for s in range(0, len(rows), chunk_rows):
        rr = rows[s:s + chunk_rows]
        h0 = splitmix64(_counters(seed, n, rr, 0))
        top = (h0 >> np.uint64(40)).astype(np.float64)
        if kind == KIND_UNIT:
            w = ((top + 1.0) * 2.0 ** -24).astype(np.float32)
        elif kind == KIND_ONE_TWO:
            w = (1.0 + top * 2.0 ** -24).astype(np.float32)
        else:
            raise ValueError("unknown weight kind")
        m = _edge_mask(seed, n, rr, p)
        blk = np.where(m, w, np.float32(np.inf))
        blk[np.arange(len(rr)), rr] = 0.0
        out[s:s + chunk_rows] = blk
    return out


def dense_graph_i64(n: int, seed: int, p: float, lo: int, hi: int,
                    inf: int = INF_I64, rows=None, chunk_rows: int = 1024) -> np.ndarray:
    """Directed graph with int64 weights uniform in [lo, hi]; returns rows x n."""
    rows = np.arange(n) if rows is None else np.asarray(rows)
    out = np.empty((len(rows), n), dtype=np.int64)
    span = np.uint64(hi - lo + 1)
    for s in range(0, len(rows), chunk_rows):
        rr = rows[s:s + chunk_rows]
        h0 = splitmix64(_counters(seed, n, rr, 0))
        w = np.int64(lo) + (h0 % span).astype(np.int64)
        m = _edge_mask(seed, n, rr, p)
        blk = np.where(m, w, np.int64(inf))
        blk[np.arange(len(rr)), rr] = 0
        out[s:s + chunk_rows] = blk
    return out


def dense_graph_f64(n: int, seed: int, p: float, kind: int = KIND_UNIT,
                    rows=None, chunk_rows: int = 1024) -> np.ndarray:
    """Directed graph with fp64 weights (full 53-bit mantissas) in (0,1]
    (KIND_UNIT) or [1,2) (KIND_ONE_TWO)."""
    rows = np.arange(n) if rows is None else np.asarray(rows)
    out = np.empty((len(rows), n), dtype=np.float64)
    for s in range(0, len(rows), chunk_rows):
        rr = rows[s:s + chunk_rows]
        h0 = splitmix64(_counters(seed, n, rr, 0))
        if kind == KIND_UNIT:
            w = ((h0 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        elif kind == KIND_ONE_TWO:
            w = 1.0 + (h0 >> np.uint64(12)).astype(np.float64) * 2.0 ** -52
        else:
            raise ValueError("unknown weight kind")
        m = _edge_mask(seed, n, rr, p)
        blk = np.where(m, w, np.inf)
        blk[np.arange(len(rr)), rr] = 0.0
        out[s:s + chunk_rows] = blk
    return out


def batch_sizes(seed: int, batch: int, lo: int = 64, hi: int = 2048) -> np.ndarray:
    """Vertex counts of a batch, uniform in [lo, hi]: lo + h(seed, b, 0, 0) mod (hi-lo+1)."""
    b = np.arange(batch, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = splitmix64(np.uint64(seed) * GAMMA + (b << np.uint64(1)))
    return (lo + (h % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


def normal_f32(shape, seed: int) -> np.ndarray:
    """Standard normal samples from counters via the Box-Muller transform (fp64, cast to fp32)."""
    cnt = int(np.prod(shape))
    k = np.arange(cnt, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(seed) * GAMMA
        h1 = splitmix64(base + (k << np.uint64(1)))
        h2 = splitmix64(base + ((k << np.uint64(1)) | np.uint64(1)))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53   # (0, 1]
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53           # [0, 1)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z.astype(np.float32).reshape(shape)


def adjoint_for(dist: np.ndarray, seed: int) -> np.ndarray:
    """dL/dD ~ N(0,1) on reachable off-diagonal pairs and 0 elsewhere."""
    g = normal_f32(dist.shape, seed)
    if dist.dtype.kind == "f":
        reach = np.isfinite(dist)
    else:
        reach = dist < (INF_I64 if dist.dtype == np.int64 else INF_I32)
    reach = reach.copy()
    np.fill_diagonal(reach, False)
    return np.where(reach, g, np.float32(0.0)).astype(np.float32)
