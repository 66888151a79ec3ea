"""Python binding of libfw.so, the GB300 blocked Floyd-Warshall library.

Argument marshalling only: every step of the solve runs in the CUDA kernels of
libfw.so (see include/fw.h for the C ABI these functions mirror).  PyTorch is
used for device memory and streams.  There is no CPU fallback: importing the
binding works without a GPU, but any call fails loudly when libfw.so is
missing or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "FWError", "Options", "load", "check", "fw_solve", "fw_solve_ex", "fw_solve_host",
    "fw_solve_host_io", "fw_solve_noalloc", "fw_sync_status", "fw_backward", "fw_backward_strided",
    "fw_peak_probe", "fw_verify_certificate", "fw_release_workspace", "fw_solve_plan",
    "fw_queue_tasks", "fw_batched_task_list", "fw_paths", "fw_intermediate", "fw_tile_closure", "fw_tile_minplus", "fw_block_init_pred",
    "BatchedPlan", "fw_bs_table", "fw_autotune_bs", "padded", "solve",
    "solve_batched", "INF_I32", "INF_I64", "FW_I32", "FW_F32", "FW_I64", "FW_F64", "DRIVER_AUTO",
    "DRIVER_PERSISTENT", "DRIVER_PHASED",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfw.so")

INF_I32 = 1 << 29
INF_I64 = 1 << 61
FW_I32, FW_F32, FW_I64, FW_F64 = 0, 1, 2, 3
DRIVER_AUTO, DRIVER_PERSISTENT, DRIVER_PHASED = 0, 1, 2

STATUS = {0: "FW_OK", 1: "FW_ERR_ARG", 2: "FW_ERR_CUDA", 3: "FW_ERR_TIMEOUT",
          4: "FW_ERR_NEG_CYCLE", 5: "FW_ERR_NOMEM", 6: "FW_ERR_UNSUPPORTED"}


class FWError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s (%d)%s" % (STATUS.get(code, "?"), code, (": " + what) if what else ""))


class Options(ctypes.Structure):
    """Mirror of fw_options (include/fw.h)."""
    _fields_ = [
        ("bs", ctypes.c_int32),
        ("driver", ctypes.c_int32),
        ("lookahead", ctypes.c_int32),
        ("grid", ctypes.c_int32),
        ("timeout_ns", ctypes.c_int64),
        ("packed_keys", ctypes.c_int32),
        ("debug_skip_release", ctypes.c_int32),
        ("ev_start", ctypes.c_void_p),
        ("ev_stop", ctypes.c_void_p),
        ("trace", ctypes.c_void_p),
        ("trace_cap", ctypes.c_int64),
        ("trace_stride", ctypes.c_int32),
        ("tile_tma", ctypes.c_int32),
        ("debug_shuffle", ctypes.c_uint64),
    ]

    @classmethod
    def default(cls, **kw) -> "Options":
        o = cls()
        load().fw_options_default(ctypes.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError("unknown option %r" % k)
            setattr(o, k, v)
        return o


_lock = threading.Lock()
_lib = None


def load():
    """Load libfw.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfw.so is not built (%s); run __graft_entry__.build() or "
                               "python paper_2403_18619_gb300/build.py" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.fw_options_default.argtypes = [P]
        lib.fw_options_default.restype = None
        lib.fw_status_string.argtypes = [I32]
        lib.fw_status_string.restype = ctypes.c_char_p
        lib.fw_solve.argtypes = [P, P, I64, I64, I32, P]
        lib.fw_solve_ex.argtypes = [P, P, I64, I64, I32, P, P]
        lib.fw_solve_host.argtypes = [P, P, I64, I64, I32, P, P]
        lib.fw_solve_host_io.argtypes = [P, P, P, I64, I64, I32, P, P]
        lib.fw_batched_plan_create.argtypes = [P, P, P, I64, I32, P]
        lib.fw_solve_batched.argtypes = [P, P, P, P]
        lib.fw_batched_plan_info.argtypes = [P, P, P]
        lib.fw_batched_plan_destroy.argtypes = [P]
        lib.fw_backward.argtypes = [P, P, P, P, I64, I64, P]
        lib.fw_backward_strided.argtypes = [P, P, P, P, I64, I64, I64, I64, P]
        lib.fw_sync_status.argtypes = [P]
        lib.fw_release_workspace.argtypes = []
        lib.fw_peak_probe.argtypes = [I32, P, P, P, P]
        lib.fw_verify_certificate.argtypes = [P, P, P, I64, I64, P, P]
        lib.fw_queue_tasks.argtypes = [I32, I64, I64, I64, P]
        lib.fw_batched_task_list.argtypes = [P, P, I64, I32, P, P, I64, P]
        lib.fw_solve_plan.argtypes = [I64, I32, P, I32, P, P, P, P]
        lib.fw_paths.argtypes = [P, I64, I64, P, P, I64, P, I64, P, P]
        lib.fw_intermediate.argtypes = [P, P, I64, I64, I64, I64, P]
        lib.fw_solve_noalloc.argtypes = [P, P, I64, I64, I32, P]
        lib.fw_tile_closure.argtypes = [P, P, I64, I32, I32, P]
        lib.fw_tile_minplus.argtypes = [P, P, I64, P, I64, P, I64, P, I64, I64, I64, I32, I64,
                                        I64, I32, P]
        lib.fw_block_init_pred.argtypes = [P, P, I64, I64, I64, I32, I64, I64, I64, I64, I64,
                                           I32, P]
        lib.fw_bs_table.argtypes = [I32, P, I32]
        lib.fw_autotune_bs.argtypes = [I32, I64, I64, P, P, P]
        for name in ("fw_solve", "fw_solve_ex", "fw_solve_host", "fw_solve_host_io",
                     "fw_batched_plan_create",
                     "fw_solve_batched", "fw_batched_plan_info", "fw_batched_plan_destroy",
                     "fw_backward", "fw_backward_strided", "fw_sync_status",
                     "fw_release_workspace", "fw_peak_probe", "fw_verify_certificate",
                     "fw_queue_tasks", "fw_batched_task_list", "fw_solve_noalloc", "fw_bs_table",
                     "fw_autotune_bs",
                     "fw_solve_plan", "fw_paths", "fw_intermediate", "fw_tile_closure",
                     "fw_tile_minplus",
                     "fw_block_init_pred"):
            getattr(lib, name).restype = I32
        _lib = lib
        return lib


def check(code: int, what: str = "") -> None:
    if code != 0:
        raise FWError(code, what)


# ------------------------------------------------------------- marshalling ---

def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(t) -> int:
    import torch
    codes = {torch.int32: FW_I32, torch.float32: FW_F32, torch.int64: FW_I64,
             torch.float64: FW_F64}
    if t.dtype not in codes:
        raise TypeError("dist must be int32, float32, int64 or float64, got %s" % t.dtype)
    return codes[t.dtype]


def _matrix(t, name):
    """(pointer, n, ld) of a CUDA 2-D tensor with unit column stride."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dim() != 2 or t.shape[0] != t.shape[1] or t.stride(1) != 1:
        raise ValueError("%s must be an n x n view with unit column stride" % name)
    return t.data_ptr(), t.shape[0], t.stride(0)


def fw_solve(dist, pred, stream=None) -> None:
    """fw_solve on CUDA tensors (n x n views, leading dimension = row stride);
    pred=None solves for distances only."""
    dp, n, ld = _matrix(dist, "dist")
    pp = _pred_arg(pred, n, ld)
    check(load().fw_solve(dp, pp, n, ld, _dtype_code(dist), _stream_ptr(stream)), "fw_solve")


def _pred_arg(pred, n, ld):
    """Device pointer of pred, or None for a distance-only solve."""
    if pred is None:
        return None
    pp, n2, ld2 = _matrix(pred, "pred")
    if n2 != n or ld2 != ld:
        raise ValueError("dist and pred must have the same shape and row stride")
    return pp


def fw_solve_ex(dist, pred, options: Options | None = None, stream=None) -> None:
    """fw_solve_ex on CUDA tensors; pred=None solves for distances only."""
    dp, n, ld = _matrix(dist, "dist")
    pp = _pred_arg(pred, n, ld)
    o = ctypes.byref(options) if options is not None else None
    check(load().fw_solve_ex(dp, pp, n, ld, _dtype_code(dist), o, _stream_ptr(stream)),
          "fw_solve_ex")


def fw_solve_noalloc(dist, pred, stream=None) -> None:
    """fw_solve_noalloc on CUDA tensors: the solve without any device allocation
    (workspace in a fixed static device array; n <= 4096; synchronous)."""
    dp, n, ld = _matrix(dist, "dist")
    pp = _pred_arg(pred, n, ld)
    check(load().fw_solve_noalloc(dp, pp, n, ld, _dtype_code(dist), _stream_ptr(stream)),
          "fw_solve_noalloc")


def _host_matrix(a, name):
    """(pointer, n, ld, dtype code) of a host matrix (numpy array or CPU torch
    tensor) with unit column stride."""
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dim() != 2 or a.stride(1) != 1 or a.shape[0] != a.shape[1]:
            raise ValueError("%s must be an n x n host view with unit column stride" % name)
        return a.data_ptr(), a.shape[0], a.stride(0), _dtype_code(a)
    if a.ndim != 2 or a.strides[1] != a.itemsize or a.shape[0] != a.shape[1]:
        raise ValueError("%s must be an n x n array with unit column stride" % name)
    code = {np.dtype(np.int32): FW_I32, np.dtype(np.float32): FW_F32,
            np.dtype(np.int64): FW_I64, np.dtype(np.float64): FW_F64}.get(a.dtype)
    if code is None:
        raise TypeError("%s must be int32, float32, int64 or float64" % name)
    return a.ctypes.data, a.shape[0], a.strides[0] // a.itemsize, code


def _host_pred(pred, n, ld):
    """Pointer of a host int32 predecessor matrix (n x n, row stride ld), or
    None for a distance-only solve."""
    if pred is None:
        return None
    pp, pn, pld, pcode = _host_matrix(pred, "pred")
    if (pn, pld, pcode) != (n, ld, FW_I32):
        raise ValueError("pred must be int32 with the distances' shape and row stride")
    return pp


def fw_solve_host(dist, pred, options: Options | None = None, stream=None) -> None:
    """fw_solve_host on host arrays (numpy or pinned CPU torch tensors), synchronous:
    dist holds the weights on entry and the distances on exit."""
    dptr, n, ld, code = _host_matrix(dist, "dist")
    o = ctypes.byref(options) if options is not None else None
    check(load().fw_solve_host(dptr, _host_pred(pred, n, ld), n, ld, code, o,
                               _stream_ptr(stream)), "fw_solve_host")


def fw_solve_host_io(weights, dist, pred, options: Options | None = None, stream=None) -> None:
    """fw_solve_host_io: weights (host, left unchanged) in, distances and
    predecessors out to their own host buffers (same shape and row stride);
    synchronous."""
    wptr, n, ld, code = _host_matrix(weights, "weights")
    dptr, n2, ld2, code2 = _host_matrix(dist, "dist")
    if (n2, ld2, code2) != (n, ld, code):
        raise ValueError("dist must have the weights' shape, row stride and dtype")
    o = ctypes.byref(options) if options is not None else None
    check(load().fw_solve_host_io(wptr, dptr, _host_pred(pred, n, ld), n, ld, code, o,
                                  _stream_ptr(stream)), "fw_solve_host_io")


def fw_backward(grad_dist, dist, pred, grad_w, stream=None) -> None:
    """fw_backward on CUDA fp32 tensors (n x n views with a common row stride)."""
    gp, n, ld = _matrix(grad_dist, "grad_dist")
    dp, _, ld1 = _matrix(dist, "dist")
    pp, _, ld2 = _matrix(pred, "pred")
    wp, _, ld3 = _matrix(grad_w, "grad_w")
    if len({ld, ld1, ld2, ld3}) != 1:
        raise ValueError("all four matrices need the same row stride")
    check(load().fw_backward(gp, dp, pp, wp, n, ld, _stream_ptr(stream)), "fw_backward")


def fw_backward_strided(grad_dist, dist, pred, grad_w, stream=None) -> None:
    """fw_backward_strided on (B, n, ld) CUDA tensors viewed as (B, n, n)."""
    for t in (grad_dist, dist, pred, grad_w):
        if t.dim() != 3 or t.stride(2) != 1 or t.stride(0) != grad_dist.stride(0) or \
                t.stride(1) != grad_dist.stride(1):
            raise ValueError("expected (B, n, n) views with identical strides")
    B, n = grad_dist.shape[0], grad_dist.shape[1]
    check(load().fw_backward_strided(grad_dist.data_ptr(), dist.data_ptr(), pred.data_ptr(),
                                     grad_w.data_ptr(), n, grad_dist.stride(1), B,
                                     grad_dist.stride(0), _stream_ptr(stream)),
          "fw_backward_strided")


def fw_sync_status(stream=None) -> None:
    check(load().fw_sync_status(_stream_ptr(stream)), "device status")


def fw_release_workspace() -> None:
    check(load().fw_release_workspace(), "fw_release_workspace")


def fw_peak_probe(dtype: int = FW_I32, stream=None):
    """(relaxations/s, relaxations per SM clock, average SM MHz) at the current clocks."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(load().fw_peak_probe(dtype, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                               _stream_ptr(stream)), "fw_peak_probe")
    return a.value, b.value, c.value


def fw_verify_certificate(W, dist, pred, stream=None) -> np.ndarray:
    """GPU certificate counts [diag, tight pred, feasibility, pred domain] (int32 only)."""
    wp, n, ld = _matrix(W, "W")
    dp, _, _ = _matrix(dist, "dist")
    pp, _, _ = _matrix(pred, "pred")
    bad = np.zeros(4, np.int64)
    check(load().fw_verify_certificate(wp, dp, pp, n, ld, bad.ctypes.data, _stream_ptr(stream)),
          "fw_verify_certificate")
    return bad


def fw_paths(pred, src, dst, max_len: int, stream=None):
    """fw_paths on CUDA tensors: pred (n x n view of a solved predecessor
    matrix), src / dst (int32 vectors of vertex ids).  Returns (paths, lengths):
    paths[q, :lengths[q]] are the vertices from src[q] to dst[q]; lengths[q] is
    0 when dst[q] is unreachable and -1 for an invalid request."""
    import torch
    pp, n, ld = _matrix(pred, "pred")
    if pred.dtype != torch.int32:
        raise TypeError("pred must be int32")
    for name, v in (("src", src), ("dst", dst)):
        if not isinstance(v, torch.Tensor) or not v.is_cuda or v.dtype != torch.int32 \
                or v.dim() != 1 or not v.is_contiguous():
            raise TypeError("%s must be a contiguous int32 CUDA vector" % name)
    if src.numel() != dst.numel():
        raise ValueError("src and dst must have the same length")
    m = src.numel()
    out = torch.empty((m, max(1, int(max_len))), dtype=torch.int32, device=pred.device)
    lens = torch.empty((m,), dtype=torch.int32, device=pred.device)
    check(load().fw_paths(pp, n, ld, src.data_ptr(), dst.data_ptr(), m, out.data_ptr(),
                          int(max_len), lens.data_ptr(), _stream_ptr(stream)), "fw_paths")
    return out, lens


def fw_intermediate(pred, out=None, stream=None):
    """fw_intermediate on CUDA int32 tensors: pred an (n, n) or (B, n, n) view
    of solved last hops (unit column stride).  Returns out (a new tensor of
    pred's shape, or the given one; out=pred works in place): the largest
    intermediate vertex of each recorded path, -1 where the path has none or
    there is no path -- the k of the paper's Fig. 1 on unique shortest paths."""
    import torch
    if not isinstance(pred, torch.Tensor) or not pred.is_cuda or pred.dtype != torch.int32:
        raise TypeError("pred must be an int32 CUDA tensor")
    if pred.dim() not in (2, 3) or pred.shape[-1] != pred.shape[-2] or pred.stride(-1) != 1:
        raise ValueError("pred must be an (n, n) or (B, n, n) view with unit column stride")
    if out is None:
        out = torch.empty_strided(pred.shape, pred.stride(), dtype=torch.int32,
                                  device=pred.device)
    if out.shape != pred.shape or out.stride() != pred.stride() or out.dtype != torch.int32 \
            or out.device != pred.device:
        raise ValueError("out must be an int32 tensor with pred's shape, strides and device")
    n, ld = pred.shape[-1], pred.stride(-2)
    B = pred.shape[0] if pred.dim() == 3 else 1
    stride = pred.stride(0) if pred.dim() == 3 else n * ld
    check(load().fw_intermediate(pred.data_ptr(), out.data_ptr(), n, ld, B, stride,
                                 _stream_ptr(stream)), "fw_intermediate")
    return out


def fw_solve_plan(n: int, options: Options | None = None, sms: int = 152,
                  dtype: int = FW_I32) -> dict:
    """What fw_solve_ex would choose for n vertices of `dtype` on a GPU with
    `sms` SMs: block size, rounds, queue lookahead and device workspace bytes
    (host only)."""
    bs, rounds = ctypes.c_int32(), ctypes.c_int32()
    look, ws = ctypes.c_int64(), ctypes.c_int64()
    o = ctypes.byref(options) if options is not None else None
    check(load().fw_solve_plan(n, dtype, o, sms, ctypes.byref(bs), ctypes.byref(rounds),
                               ctypes.byref(look), ctypes.byref(ws)), "fw_solve_plan")
    return {"bs": bs.value, "rounds": rounds.value, "lookahead": look.value,
            "workspace_bytes": ws.value}


def fw_queue_tasks(R: int, lookahead: int, first: int = 0, count: int | None = None) -> np.ndarray:
    """The persistent driver's queue: rows of (type, round, tile row, tile column)."""
    if count is None:
        count = R ** 3 - first
    out = np.zeros((count, 4), np.int32)
    check(load().fw_queue_tasks(R, lookahead, first, count, out.ctypes.data), "fw_queue_tasks")
    return out


def fw_batched_task_list(ns, bss, sms: int = 152, options: Options | None = None) -> np.ndarray:
    """The claim order of a batched plan of graphs with ns[b] vertices and
    block sizes bss[b]: rows of (graph, task index in that graph's queue)."""
    ns = np.ascontiguousarray(np.asarray(ns, np.int64))
    bss = np.ascontiguousarray(np.asarray(bss, np.int32))
    if ns.shape != bss.shape or ns.ndim != 1:
        raise ValueError("ns and bss must be 1-D of equal length")
    total = int(sum(-(-int(n) // int(b)) ** 3 for n, b in zip(ns, bss)))
    out = np.zeros((max(total, 1), 2), np.int32)
    cnt = ctypes.c_int64()
    o = ctypes.byref(options) if options is not None else None
    check(load().fw_batched_task_list(ns.ctypes.data, bss.ctypes.data, len(ns), sms, o,
                                      out.ctypes.data, total, ctypes.byref(cnt)),
          "fw_batched_task_list")
    return out[:cnt.value]


def _block(t, name):
    """(pointer, rows, cols, ld) of a CUDA 2-D tensor with unit column stride."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("%s must be a 2-D view with unit column stride" % name)
    return t.data_ptr(), t.shape[0], t.shape[1], t.stride(0)


def fw_tile_closure(tile, pred, bs: int, stream=None) -> None:
    """fw_tile_closure on a bs x bs CUDA view (pred: same layout, or None)."""
    tp, r, c, ld = _block(tile, "tile")
    if r != bs or c != bs:
        raise ValueError("tile must be bs x bs")
    pp = None
    if pred is not None:
        pp, r2, c2, ld2 = _block(pred, "pred")
        if (r2, c2, ld2) != (r, c, ld):
            raise ValueError("pred must have the tile's shape and row stride")
    check(load().fw_tile_closure(tp, pp, ld, bs, _dtype_code(tile), _stream_ptr(stream)),
          "fw_tile_closure")


def fw_tile_minplus(C, Pc, A, B, Pb, bs: int, skip_tile_row: int = -1, skip_tile_col: int = -1,
                    stream=None) -> None:
    """fw_tile_minplus: C = min(C, A (x) B) tile by tile, Pc from Pb's rows
    (Pc, Pb: None for distances only).  C is (tiles_m * bs) x (tiles_n * bs);
    A is (tiles_m * bs) x bs, B and Pb are bs x (tiles_n * bs)."""
    cp, cr, cc, ldc = _block(C, "C")
    ap, ar, ac, lda = _block(A, "A")
    bp, br, bc, ldb = _block(B, "B")
    if cr % bs or cc % bs or ar != cr or ac != bs or br != bs or bc != cc:
        raise ValueError("shapes must be C (m bs x n bs), A (m bs x bs), B (bs x n bs)")
    if A.dtype != C.dtype or B.dtype != C.dtype:
        raise TypeError("A, B and C must share a dtype")
    pcp = pbp = None
    ldpb = 0
    if (Pc is None) != (Pb is None):
        raise ValueError("Pc and Pb must both be given or both be None")
    if Pc is not None:
        pcp, r2, c2, ld2 = _block(Pc, "Pc")
        if (r2, c2, ld2) != (cr, cc, ldc):
            raise ValueError("Pc must have C's shape and row stride")
        pbp, r3, c3, ldpb = _block(Pb, "Pb")
        if (r3, c3) != (bs, cc):
            raise ValueError("Pb must be bs x (tiles_n * bs)")
    check(load().fw_tile_minplus(cp, pcp, ldc, ap, lda, bp, ldb, pbp, ldpb, cr // bs, cc // bs,
                                 bs, skip_tile_row, skip_tile_col, _dtype_code(C),
                                 _stream_ptr(stream)), "fw_tile_minplus")


def fw_block_init_pred(dist, pred, bs: int, n: int, row_tile0: int, row_tile_step: int,
                       col_tile0: int, col_tile_step: int, stream=None) -> None:
    """fw_block_init_pred on a local block (CUDA views with one row stride)."""
    dp, r, c, ld = _block(dist, "dist")
    pp, r2, c2, ld2 = _block(pred, "pred")
    if (r2, c2, ld2) != (r, c, ld):
        raise ValueError("pred must have dist's shape and row stride")
    check(load().fw_block_init_pred(dp, pp, ld, r, c, bs, n, row_tile0, row_tile_step,
                                    col_tile0, col_tile_step, _dtype_code(dist),
                                    _stream_ptr(stream)), "fw_block_init_pred")


class BatchedPlan:
    """fw_batched_plan_create / fw_solve_batched / fw_batched_plan_destroy."""

    def __init__(self, ns, lds, dtype: int = FW_I32, options: Options | None = None):
        lib = load()
        ns = np.ascontiguousarray(np.asarray(ns, np.int64))
        lds = np.ascontiguousarray(np.asarray(lds, np.int64))
        if ns.shape != lds.shape or ns.ndim != 1:
            raise ValueError("ns and lds must be 1-D of equal length")
        self.batch = len(ns)
        self._h = ctypes.c_void_p()
        o = ctypes.byref(options) if options is not None else None
        check(lib.fw_batched_plan_create(ctypes.byref(self._h), ns.ctypes.data, lds.ctypes.data,
                                         self.batch, dtype, o), "fw_batched_plan_create")
        self._dp = (ctypes.c_void_p * self.batch)()
        self._pp = (ctypes.c_void_p * self.batch)()

    def solve(self, dists, preds, stream=None) -> None:
        """dists/preds: sequences of CUDA tensors (n_b x n_b views) or raw device
        pointers; preds=None solves every graph for distances only."""
        if len(dists) != self.batch or (preds is not None and len(preds) != self.batch):
            raise ValueError("expected %d graphs" % self.batch)
        for b, d in enumerate(dists):
            self._dp[b] = d if isinstance(d, int) else d.data_ptr()
        if preds is not None:
            for b, p in enumerate(preds):
                self._pp[b] = p if isinstance(p, int) else p.data_ptr()
        check(load().fw_solve_batched(self._h, self._dp, self._pp if preds is not None else None,
                                      _stream_ptr(stream)), "fw_solve_batched")

    def info(self):
        bs = np.zeros(self.batch, np.int32)
        tot = ctypes.c_int64()
        check(load().fw_batched_plan_info(self._h, bs.ctypes.data, ctypes.byref(tot)),
              "fw_batched_plan_info")
        return bs, tot.value

    def close(self) -> None:
        if self._h:
            load().fw_batched_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fw_bs_table(table=None, dtype: int = FW_I32) -> np.ndarray:
    """Read (table=None) or set dtype's 7-entry per-size-class block-size table."""
    t = np.zeros(7, np.int32) if table is None else np.ascontiguousarray(table, np.int32)
    check(load().fw_bs_table(dtype, t.ctypes.data, 0 if table is None else 1), "fw_bs_table")
    return t


def fw_autotune_bs(dtype: int = FW_I32, graphs_per_class: int = 32, max_n: int = 2048,
                   stream=None):
    """Measure and install the per-size-class block sizes; returns (table, best ms)."""
    t = np.zeros(7, np.int32)
    ms = np.zeros(7, np.float64)
    check(load().fw_autotune_bs(dtype, graphs_per_class, max_n, _stream_ptr(stream),
                                t.ctypes.data, ms.ctypes.data), "fw_autotune_bs")
    return t, ms


# ------------------------------------------------------------ convenience ---

def padded(n: int) -> int:
    """Smallest leading dimension >= n that keeps rows 16-byte aligned."""
    return (n + 3) // 4 * 4


def solve_batched(Ws, options: Options | None = None, stream=None, sync: bool = True):
    """Out-of-place batched solve of CUDA weight matrices: returns [(D, P), ...]."""
    import torch
    Ds, Ps, ns, lds = [], [], [], []
    for W in Ws:
        n = W.shape[0]
        ld = padded(n)
        Dbuf = torch.empty((n, ld), dtype=W.dtype, device=W.device)
        Pbuf = torch.empty((n, ld), dtype=torch.int32, device=W.device)
        Dbuf[:, :n].copy_(W)
        Ds.append(Dbuf[:, :n])
        Ps.append(Pbuf[:, :n])
        ns.append(n)
        lds.append(ld)
    plan = BatchedPlan(ns, lds, _dtype_code(Ws[0]), options)
    plan.solve(Ds, Ps, stream)
    if sync:
        fw_sync_status(stream)
    plan.close()
    return list(zip(Ds, Ps))


def solve(W, options: Options | None = None, stream=None, sync: bool = True,
          with_pred: bool = True):
    """Out-of-place solve of a CUDA n x n weight matrix: returns (D, P) views
    (P is None when with_pred is False: a distance-only solve)."""
    import torch
    n = W.shape[0]
    ld = padded(n)
    Dbuf = torch.empty((n, ld), dtype=W.dtype, device=W.device)
    D = Dbuf[:, :n]
    P = None
    if with_pred:
        P = torch.empty((n, ld), dtype=torch.int32, device=W.device)[:, :n]
    D.copy_(W)
    fw_solve_ex(D, P, options, stream)
    if sync:
        fw_sync_status(stream)
    return D, P
