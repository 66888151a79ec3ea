"""CPU oracle for blocked Floyd-Warshall: TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library (the CUDA path and
its Python binding) never imports, links or calls it, and the two share no code.

The arithmetic lives in ``fw_oracle.c`` (plain loops in int64 / fp64, each
function citing the definition it writes out); this module compiles it with gcc
on first use and wraps it for numpy arrays.

What each function is pinned to (tests/test_oracle.py):
  fw_i64 / fw_f64          Dijkstra from every source, scipy's shortest_path
                           (distances and last-hop predecessors), brute-force
                           enumeration of simple paths (n <= 7), closed forms
                           (path, ring, unit complete graph, disconnected).
  dijkstra_*               scipy's dijkstra.
  certificate_i64          hand-built correct/incorrect inputs (planted faults).
  path_count_i64           brute-force enumeration of shortest paths.
  grad_f64                 central finite differences of the fp64 oracle.
  fw_k_i64 / fw_k_f64      brute-force enumeration of shortest simple paths
                           (smallest largest-intermediate over them), closed
                           forms (paths numbered up and down).
  max_intermediate         brute-force enumeration on unique-path graphs, and
                           fw_k_* on every pair with a unique shortest path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF_I32 = 1 << 29
INF_I64 = 1 << 61


def build(force: bool = False) -> str:
    """Compile fw_oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int64
            lib.oracle_fw_i64.argtypes = [P, I, I, P, P, ctypes.c_int]
            lib.oracle_fw_f64.argtypes = [P, I, P, P, ctypes.c_int]
            lib.oracle_dijkstra_i64.argtypes = [P, I, I, P, I, P, P, ctypes.c_int]
            lib.oracle_dijkstra_f64.argtypes = [P, I, P, I, P, P, ctypes.c_int]
            lib.oracle_certificate_i64.argtypes = [P, P, P, I, I, P, I, P, ctypes.c_int]
            lib.oracle_path_count_i64.argtypes = [P, P, I, I, P, I, P, ctypes.c_int]
            lib.oracle_lasthop_margin_f64.argtypes = [P, P, P, I, P, I, P, ctypes.c_int]
            lib.oracle_lasthop_margin_i64.argtypes = [P, P, P, I, I, P, I, P, ctypes.c_int]
            lib.oracle_hops.argtypes = [P, I, P, I, P, ctypes.c_int]
            lib.oracle_fw_k_i64.argtypes = [P, I, I, P, P, ctypes.c_int]
            lib.oracle_fw_k_f64.argtypes = [P, I, P, P, ctypes.c_int]
            lib.oracle_max_intermediate.argtypes = [P, I, P, I, P, ctypes.c_int]
            lib.oracle_grad_f64.argtypes = [P, P, I, P]
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _rows(rows, n):
    if rows is None:
        return None, None, n
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    return r, r.ctypes.data, len(r)


def threads_default() -> int:
    return int(os.environ.get("ORACLE_THREADS", "0"))


def fw_i64(W: np.ndarray, inf: int | None = None, threads: int | None = None):
    """Plain FW (Fig. 1) on int32 or int64 weights in int64: returns (D int64,
    P int32).  inf defaults to 2**29 for int32 weights and 2**61 for int64."""
    lib = _load()
    n = W.shape[0]
    if inf is None:
        inf = INF_I64 if np.asarray(W).dtype == np.int64 else INF_I32
    W, wp = _c(W, np.int64)
    D = np.empty((n, n), np.int64)
    P = np.empty((n, n), np.int32)
    lib.oracle_fw_i64(wp, n, inf, D.ctypes.data, P.ctypes.data,
                      threads_default() if threads is None else threads)
    return D, P


def fw_f64(W: np.ndarray, threads: int | None = None):
    """Plain FW (Fig. 1) on fp32 or fp64 weights in fp64: returns (D float64, P int32)."""
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.float64)
    D = np.empty((n, n), np.float64)
    P = np.empty((n, n), np.int32)
    lib.oracle_fw_f64(wp, n, D.ctypes.data, P.ctypes.data,
                      threads_default() if threads is None else threads)
    return D, P


def fw_k_i64(W: np.ndarray, inf: int | None = None, threads: int | None = None):
    """Fig. 1 with its path bookkeeping P_ij <- k (strict "<"): returns (D
    int64, K int32), K[i][j] = the smallest over shortest i -> j paths of the
    largest intermediate vertex, -1 where no relaxation improved (i, j)."""
    lib = _load()
    n = W.shape[0]
    if inf is None:
        inf = INF_I64 if np.asarray(W).dtype == np.int64 else INF_I32
    W, wp = _c(W, np.int64)
    D = np.empty((n, n), np.int64)
    K = np.empty((n, n), np.int32)
    lib.oracle_fw_k_i64(wp, n, inf, D.ctypes.data, K.ctypes.data,
                        threads_default() if threads is None else threads)
    return D, K


def fw_k_f64(W: np.ndarray, threads: int | None = None):
    """fw_k_i64 for real weights, in fp64: returns (D float64, K int32)."""
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.float64)
    D = np.empty((n, n), np.float64)
    K = np.empty((n, n), np.int32)
    lib.oracle_fw_k_f64(wp, n, D.ctypes.data, K.ctypes.data,
                        threads_default() if threads is None else threads)
    return D, K


def max_intermediate(Prows, rows=None, threads=None):
    """Largest intermediate vertex on each path a last-hop matrix records (-1:
    diagonal, single edge, unreachable, or P not leading back to the source)."""
    lib = _load()
    P, pp = _c(Prows, np.int32)
    n = P.shape[1]
    r, rp, m = _rows(rows, n)
    out = np.empty((m, n), np.int32)
    lib.oracle_max_intermediate(pp, n, rp, m, out.ctypes.data,
                                threads_default() if threads is None else threads)
    return out


def dijkstra_i64(W, sources, inf: int = INF_I32, threads: int | None = None):
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.int32)
    s, sp, m = _rows(sources, n)
    D = np.empty((m, n), np.int64)
    P = np.empty((m, n), np.int32)
    lib.oracle_dijkstra_i64(wp, n, inf, sp, m, D.ctypes.data, P.ctypes.data,
                            threads_default() if threads is None else threads)
    return D, P


def dijkstra_f64(W, sources, threads: int | None = None):
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.float32)
    s, sp, m = _rows(sources, n)
    D = np.empty((m, n), np.float64)
    P = np.empty((m, n), np.int32)
    lib.oracle_dijkstra_f64(wp, n, sp, m, D.ctypes.data, P.ctypes.data,
                            threads_default() if threads is None else threads)
    return D, P


def certificate_i64(W, Drows, Prows, rows=None, inf: int = INF_I32, threads=None):
    """Counts of violated certificate conditions [diag, tight-pred, feasibility, pred-walk]."""
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.int32)
    D, dp = _c(Drows, np.int32)
    P, pp = _c(Prows, np.int32)
    r, rp, m = _rows(rows, n)
    bad = np.zeros(4, np.int64)
    lib.oracle_certificate_i64(wp, dp, pp, n, inf, rp, m, bad.ctypes.data,
                               threads_default() if threads is None else threads)
    return bad


def path_count_i64(W, Drows, rows=None, inf: int = INF_I32, threads=None):
    """Number of shortest paths per pair, capped at 2 (1 = unique)."""
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.int32)
    D, dp = _c(Drows, np.int64)
    r, rp, m = _rows(rows, n)
    cnt = np.empty((m, n), np.uint8)
    lib.oracle_path_count_i64(wp, dp, n, inf, rp, m, cnt.ctypes.data,
                              threads_default() if threads is None else threads)
    return cnt


def lasthop_margin_f64(W, Drows, Prows, rows=None, threads=None):
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.float32)
    D, dp = _c(Drows, np.float64)
    P, pp = _c(Prows, np.int32)
    r, rp, m = _rows(rows, n)
    out = np.empty((m, n), np.float64)
    lib.oracle_lasthop_margin_f64(wp, dp, pp, n, rp, m, out.ctypes.data,
                                  threads_default() if threads is None else threads)
    return out


def lasthop_margin_i64(W, Drows, Prows, rows=None, inf: int = INF_I32, threads=None):
    lib = _load()
    n = W.shape[0]
    W, wp = _c(W, np.int32)
    D, dp = _c(Drows, np.int64)
    P, pp = _c(Prows, np.int32)
    r, rp, m = _rows(rows, n)
    out = np.empty((m, n), np.int64)
    lib.oracle_lasthop_margin_i64(wp, dp, pp, n, inf, rp, m, out.ctypes.data,
                                  threads_default() if threads is None else threads)
    return out


def hops(Prows, rows=None, threads=None):
    lib = _load()
    P, pp = _c(Prows, np.int32)
    n = P.shape[1]
    r, rp, m = _rows(rows, n)
    out = np.empty((m, n), np.int32)
    lib.oracle_hops(pp, n, rp, m, out.ctypes.data,
                    threads_default() if threads is None else threads)
    return out


def grad_f64(G, P):
    """dL/dW for L = sum G * D through the last-hop trees P (fp64)."""
    lib = _load()
    n = P.shape[0]
    G, gp = _c(G, np.float64)
    P, pp = _c(P, np.int32)
    GW = np.zeros((n, n), np.float64)
    lib.oracle_grad_f64(gp, pp, n, GW.ctypes.data)
    return GW
