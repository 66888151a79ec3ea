"""Device copy of the seeded generator (graphgen_dev.cu -> libgraphgen.so).

Fills CUDA tensors with exactly the values graphgen.dense_graph_* produce on
the host; used for inputs too large to draw on the host quickly.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "graphgen_dev.cu")
LIB = os.path.join(HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-shared", "-Xcompiler", "-fPIC", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libgraphgen.so is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB)
        P, I64 = ctypes.c_void_p, ctypes.c_int64
        lib.graphgen_fill_i32.argtypes = [P, I64, I64, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P]
        lib.graphgen_fill_f32.argtypes = [P, I64, I64, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_int, P]
        lib.graphgen_fill_i64.argtypes = [P, I64, I64, ctypes.c_uint64, ctypes.c_double,
                                          I64, I64, I64, P]
        lib.graphgen_fill_f64.argtypes = [P, I64, I64, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_int, P]
        _lib = lib
    return _lib


def _stream(stream):
    import torch
    return (stream or torch.cuda.current_stream()).cuda_stream


def fill_i32(t, seed: int, p: float, lo: int, hi: int, inf: int = 1 << 29, stream=None):
    n, ld = t.shape[0], t.stride(0)
    rc = _load().graphgen_fill_i32(t.data_ptr(), n, ld, seed, p, lo, hi, inf, _stream(stream))
    if rc:
        raise RuntimeError("graphgen_fill_i32 failed (%d)" % rc)
    return t


def fill_f32(t, seed: int, p: float, kind: int = 0, stream=None):
    n, ld = t.shape[0], t.stride(0)
    rc = _load().graphgen_fill_f32(t.data_ptr(), n, ld, seed, p, kind, _stream(stream))
    if rc:
        raise RuntimeError("graphgen_fill_f32 failed (%d)" % rc)
    return t


def fill_i64(t, seed: int, p: float, lo: int, hi: int, inf: int = 1 << 61, stream=None):
    n, ld = t.shape[0], t.stride(0)
    rc = _load().graphgen_fill_i64(t.data_ptr(), n, ld, seed, p, lo, hi, inf, _stream(stream))
    if rc:
        raise RuntimeError("graphgen_fill_i64 failed (%d)" % rc)
    return t


def fill_f64(t, seed: int, p: float, kind: int = 0, stream=None):
    n, ld = t.shape[0], t.stride(0)
    rc = _load().graphgen_fill_f64(t.data_ptr(), n, ld, seed, p, kind, _stream(stream))
    if rc:
        raise RuntimeError("graphgen_fill_f64 failed (%d)" % rc)
    return t
