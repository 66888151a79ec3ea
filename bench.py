"""Benchmark: blocked Floyd-Warshall on one GB300 (or N replicas).

One step = one full all-pairs solve (distances + last-hop predecessors) of the
n = 32768 complete digraph with int32 weights uniform in [1, 10^4] and 10% of
the edges removed (INF = 2^29): 8 GiB of dist + pred in HBM, n^3 = 3.5e13
relaxations.  The metric is relaxations per second, n^3 / t.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` times the solve with the input already in HBM
(the input is restored from a pristine device copy before every step, outside
the timed events); `e2e` times fw_solve_host_io (the weights from one pinned
host buffer, the results into others), copies included.  `roofline` compares the persistent solver kernel against the
min-plus relaxation peak measured by fw_peak_probe in the same process.  The
CPU baseline is the oracle's plain triple loop on a bounded sample of the same
workload.  With --impl reference the oracle alone is timed the same way.
Under torchrun every rank solves its own instance (independent replicas; the
path has no exchange step) and rank 0 reports the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_FULL = 32768
SEED = 3
P_EDGE = 0.9
LO, HI = 1, 10_000
BS = 128
SAMPLE_N = 2048          # CPU baseline: leading 2048-vertex induced subgraph
# DRAM bytes (read + write) of one k_persistent_ws launch of the current
# kernel, keyed by (n, BS, driver); null in the line where no capture exists.
# n = 32768: one ncu capture of the same kernel at n = 16384 (339.4e9 B)
# scaled by n^3; an upper bound, since the bytes above the algorithmic
# 8 n^3 / BS (2.20e12 B here) are scattered predecessor stores whose share
# falls as n grows (1.29x at n = 8192, 1.23x at n = 16384).
TRAFFIC_BYTES = {(32768, 128, 1): 339.4e9 * 8}
TRAFFIC_NOTE = {(32768, 128, 1): "ncu dram bytes of one launch at n = 16384, scaled by n^3 "
                                 "(upper bound; algorithmic 8 n^3 / BS = 2.20e12 B)"}


def workload_name(n=N_FULL):
    return ("blocked FW, n=%d complete digraph minus 10%% edges, int32 weights U[1,1e4], "
            "INF=2^29, dist+pred (flag-scheduled persistent driver)" % n)


# ------------------------------------------------------------------ clocks ---

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------- CPU baseline ---

def cpu_baseline(budget_s: float = 20.0):
    """The oracle's plain FW on the leading SAMPLE_N vertices of the same graph."""
    import numpy as np
    import graphgen
    import oracle
    W = graphgen.dense_graph_i32(N_FULL, SEED, P_EDGE, LO, HI, rows=np.arange(SAMPLE_N))
    W = np.ascontiguousarray(W[:, :SAMPLE_N])
    threads = int(os.environ.get("ORACLE_THREADS", "0")) or (os.cpu_count() or 1)
    runs, t_total = 0, 0.0
    while True:
        t0 = time.perf_counter()
        oracle.fw_i64(W, threads=threads)
        t_total += time.perf_counter() - t0
        runs += 1
        if t_total > budget_s / 2 or runs >= 3:
            break
    t = t_total / runs
    return {"value": SAMPLE_N ** 3 / t, "unit": "relax/s", "cores": threads, "kind": "oracle",
            "sample": "plain FW triple loop (int64, OpenMP over rows) on the leading %d-vertex "
                      "induced subgraph of the same seeded graph, %d run(s), %.2f s each"
                      % (SAMPLE_N, runs, t)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import graphgen
    import oracle
    W = graphgen.dense_graph_i32(N_FULL, SEED, P_EDGE, LO, HI, rows=np.arange(SAMPLE_N))
    W = np.ascontiguousarray(W[:, :SAMPLE_N])
    threads = int(os.environ.get("ORACLE_THREADS", "0")) or (os.cpu_count() or 1)
    for _ in range(args.warmup):
        oracle.fw_i64(W, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fw_i64(W, threads=threads)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = SAMPLE_N ** 3 / t
    line = {
        "impl": "reference", "metric": "relaxations/s (n^3/t)", "value": v, "unit": "relax/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": workload_name(), "sample_n": SAMPLE_N},
        "cpu_baseline": {"value": v, "unit": "relax/s", "cores": threads, "kind": "oracle",
                         "sample": "leading %d-vertex induced subgraph per step" % SAMPLE_N},
        "e2e": {"value": v, "unit": "relax/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------- across ranks ---

def reduce_max(x: float, world: int, device="cuda") -> float:
    """Maximum of x over the ranks (x itself when there is one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def step_stats(ms) -> dict:
    """Mean, median, min and max of this rank's timed steps (ms), the spread
    behind the single rate of the line."""
    ms = [float(x) for x in ms]
    return {"mean": statistics.fmean(ms), "median": statistics.median(ms), "min": min(ms),
            "max": max(ms), "n": len(ms)}


def whole_job_rate(units_per_rank: float, world: int, t_max_s: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank runs the same workload on its own instance)."""
    return world * units_per_rank / t_max_s


# ------------------------------------------------------------------- GPU ---

def _events(k):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(k)]


def _batched_inputs(fw):
    """The 512-graph workload: n uniform in [64, 2048] (seed 11), p = 0.3,
    int32 weights in [1, 100]; inputs W and output buffers D, P per graph."""
    import torch
    import graphgen
    import graphgen.device as gdev
    ns = graphgen.batch_sizes(11, 512, 64, 2048)
    W, D, P = [], [], []
    for b, n in enumerate(ns):
        n = int(n)
        ld = fw.padded(n)
        w = torch.empty((n, ld), dtype=torch.int32, device="cuda")
        gdev.fill_i32(w[:, :n], seed=11000 + b, p=0.3, lo=1, hi=100)
        W.append(w)
        D.append(torch.empty_like(w))
        P.append(torch.empty_like(w))
    return ns, W, D, P


def trace_batched(fw, out_path):
    """One traced batched solve of the 512-graph workload (autotuned block
    sizes, every task traced): writes tracing.summarize_batched as JSON."""
    import torch
    from paper_2403_18619_gb300 import tracing
    fw.fw_autotune_bs(fw.FW_I32, graphs_per_class=16, max_n=2048)
    ns, W, D, P = _batched_inputs(fw)
    lds = [fw.padded(int(n)) for n in ns]
    probe = fw.BatchedPlan([int(n) for n in ns], lds, fw.FW_I32)
    bsv, ntasks = probe.info()
    probe.close()
    tr = torch.zeros((ntasks, 10), dtype=torch.int64, device="cuda")
    opt = fw.Options.default(trace=tr.data_ptr(), trace_cap=ntasks, trace_stride=1)
    plan = fw.BatchedPlan([int(n) for n in ns], lds, fw.FW_I32, opt)
    Dv = [d[:, :int(n)] for d, n in zip(D, ns)]
    Pv = [p_[:, :int(n)] for p_, n in zip(P, ns)]
    for _ in range(2):  # the second solve is the one kept (warm)
        for d, w in zip(D, W):
            d.copy_(w)
        tr.zero_()
        plan.solve(Dv, Pv)
        fw.fw_sync_status()
    plan.close()
    s = tracing.summarize_batched(tr.cpu().numpy(), [int(n) for n in ns], bsv.tolist())
    s["workload"] = "512 digraphs, n ~ U[64,2048] (seed 11), p=0.3, int32 U[1,100]"
    s["bs_table"] = fw.fw_bs_table().tolist()
    with open(out_path, "w") as f:
        json.dump(s, f, indent=1)
    print(json.dumps({"trace_summary": out_path, "tasks": s.get("tasks"),
                      "busy_fraction": s.get("busy_fraction")}), flush=True)


def bench_batched(fw, args):
    """512 digraphs, n uniform in [64, 2048], p = 0.3, int32 weights in [1, 100]:
    one batched launch (CUDA-graph replay) vs one fw_solve launch per graph."""
    import numpy as np
    import torch
    table, tune_ms = fw.fw_autotune_bs(fw.FW_I32, graphs_per_class=16, max_n=2048)
    ns, W, D, P = _batched_inputs(fw)
    plan = fw.BatchedPlan([int(n) for n in ns], [fw.padded(int(n)) for n in ns], fw.FW_I32)
    bsv, ntasks = plan.info()
    Dv = [d[:, :int(n)] for d, n in zip(D, ns)]
    Pv = [p_[:, :int(n)] for p_, n in zip(P, ns)]

    def restore():
        for d, w in zip(D, W):
            d.copy_(w)

    for _ in range(2):
        restore()
        plan.solve(Dv, Pv)
    fw.fw_sync_status()
    steps = max(2, args.steps)
    e0, e1 = _events(steps), _events(steps)
    for i in range(steps):
        restore()
        e0[i].record()
        plan.solve(Dv, Pv)
        e1[i].record()
    fw.fw_sync_status()
    t_batched = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / steps
    # one launch per graph, same buffers, same stream
    restore()
    for d, p_ in zip(Dv, Pv):
        fw.fw_solve(d, p_)
    fw.fw_sync_status()
    restore()
    a, b = _events(1)[0], _events(1)[0]
    a.record()
    for d, p_ in zip(Dv, Pv):
        fw.fw_solve(d, p_)
    b.record()
    fw.fw_sync_status()
    t_single = a.elapsed_time(b)
    plan.close()
    relax = float(sum(int(n) ** 3 for n in ns))
    peak = fw.fw_peak_probe(fw.FW_I32)[0]
    return {"workload": "512 digraphs, n ~ U[64,2048] (seed 11), p=0.3, int32 U[1,100]",
            "graphs_per_s": 512 / (t_batched * 1e-3), "relax_per_s": relax / (t_batched * 1e-3),
            "frac_of_peak": relax / (t_batched * 1e-3) / peak, "peak_relax_per_s": peak,
            "ms": t_batched, "one_launch_per_graph_ms": t_single,
            "speedup_vs_one_launch_per_graph": t_single / t_batched,
            "bs_table": table.tolist(), "tasks": int(ntasks),
            "timing": "events around fw_solve_batched (graph replay); inputs restored outside"}


def _peaks():
    """Measured copy bandwidth of the GB300s (driver-written), GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Algorithmic bytes per (source i, vertex v) of the backward: the row kernel
# reads dL/dD and pred and writes E; the column kernel reads pred and E and
# writes dL/dW (4 bytes each).
BWD_BYTES_PER_ENTRY = 24


def bench_backward(fw, args):
    """64 digraphs, n = 1024, p = 0.1, fp32 weights in [1, 2): batched forward +
    strided backward through the C ABI, the same through FWFunction (the call a
    training step makes; stored and recompute modes), and one forward and one
    backward launch per graph."""
    import numpy as np
    import torch
    import graphgen.device as gdev
    from paper_2403_18619_gb300.autograd import clear_plan_cache, shortest_paths
    B, n = 64, 1024
    # the fp32 block sizes of this GPU (size classes up to n)
    bs_table, _ = fw.fw_autotune_bs(fw.FW_F32, graphs_per_class=16, max_n=n)
    W = torch.empty((B, n, n), dtype=torch.float32, device="cuda")
    for b in range(B):
        gdev.fill_f32(W[b], seed=500 + b, p=0.1, kind=1)
    D = torch.empty_like(W)
    P = torch.empty((B, n, n), dtype=torch.int32, device="cuda")
    G = torch.randn((B, n, n), generator=torch.Generator(device="cuda").manual_seed(7),
                    device="cuda")
    GW = torch.empty_like(W)
    plan = fw.BatchedPlan([n] * B, [n] * B, fw.FW_F32)
    Dl = [D[b] for b in range(B)]
    Pl = [P[b] for b in range(B)]
    for _ in range(2):
        D.copy_(W)
        plan.solve(Dl, Pl)
        fw.fw_backward_strided(G, D, P, GW)
    fw.fw_sync_status()
    steps = max(3, args.steps)
    f0, f1, b1 = _events(steps), _events(steps), _events(steps)
    for i in range(steps):
        D.copy_(W)
        f0[i].record()
        plan.solve(Dl, Pl)
        f1[i].record()
        fw.fw_backward_strided(G, D, P, GW)
        b1[i].record()
    fw.fw_sync_status()
    fwd = sum(a.elapsed_time(b) for a, b in zip(f0, f1)) / steps
    bwd = sum(a.elapsed_time(b) for a, b in zip(f1, b1)) / steps
    D.copy_(W)
    a, b = _events(1)[0], _events(1)[0]
    a.record()
    for g in range(B):
        fw.fw_solve(D[g], P[g])
        fw.fw_backward(G[g], D[g], P[g], GW[g])
    b.record()
    fw.fw_sync_status()
    t_single = a.elapsed_time(b)
    plan.close()

    # the user's path: FWFunction forward (copy of W, batched solve) and backward
    def autograd_ms(recompute):
        Wt = W.detach().requires_grad_(True)
        for _ in range(2):
            Dt, _ = shortest_paths(Wt, recompute=recompute)
            torch.autograd.backward(Dt, grad_tensors=G)
            Wt.grad = None
        ts = []
        for _ in range(steps):
            e0, e1 = _events(2)
            e0.record()
            Dt, _ = shortest_paths(Wt, recompute=recompute)
            torch.autograd.backward(Dt, grad_tensors=G)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            Wt.grad = None
            del Dt
        return sum(ts) / len(ts)

    ag = autograd_ms(False)
    ag_rec = autograd_ms(True)
    clear_plan_cache()
    hbm, src = _peaks()
    algo = float(B) * n * n * BWD_BYTES_PER_ENTRY
    return {"workload": "64 digraphs, n=1024, p=0.1, fp32 U[1,2), dL/dD ~ N(0,1)",
            "bs_table_f32": bs_table.tolist(),
            "bwd_ms": bwd, "fwd_ms": fwd, "fwd_bwd_ms": fwd + bwd,
            "bwd_roofline": {"bound": "hbm", "algorithmic_bytes": algo,
                             "bytes_per_entry": BWD_BYTES_PER_ENTRY,
                             "achieved_gbs": algo / (bwd * 1e-3) / 1e9, "peak_gbs": hbm,
                             "frac": algo / (bwd * 1e-3) / 1e9 / hbm,
                             "peak_source": "%s copy bandwidth" % src},
            "autograd_fwd_bwd_ms": ag, "autograd_recompute_fwd_bwd_ms": ag_rec,
            "autograd_over_raw": ag / (fwd + bwd),
            "one_launch_per_graph_fwd_bwd_ms": t_single,
            "speedup_vs_one_launch_per_graph": t_single / (fwd + bwd)}


# Algorithmic bytes per entry of fw_intermediate: read pred, write the result.
MID_BYTES_PER_ENTRY = 8


def bench_intermediate(fw, args):
    """fw_intermediate (the paper's P_ij = k bookkeeping from last hops) on the
    predecessors of an 8192-vertex int32 solve (p = 0.5, weights U[1, 100])."""
    import torch
    import graphgen.device as gdev
    n = 8192
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    P = torch.empty_like(D)
    gdev.fill_i32(D, seed=8192, p=0.5, lo=1, hi=100)
    fw.fw_solve(D, P)
    out = torch.empty_like(P)
    for _ in range(3):
        fw.fw_intermediate(P, out=out)
    fw.fw_sync_status()
    steps = max(5, args.steps)
    ev = _events(steps + 1)
    ev[0].record()
    for i in range(steps):
        fw.fw_intermediate(P, out=out)   # 512 MB in, 256 MB written: larger than L2
        ev[i + 1].record()
    torch.cuda.synchronize()
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    avg = sum(ms) / steps
    hbm, src = _peaks()
    algo = float(n) * n * MID_BYTES_PER_ENTRY
    return {"workload": "pred of an 8192-vertex int32 solve, p=0.5", "ms": avg,
            "roofline": {"bound": "hbm", "algorithmic_bytes": algo,
                         "bytes_per_entry": MID_BYTES_PER_ENTRY,
                         "achieved_gbs": algo / (avg * 1e-3) / 1e9, "peak_gbs": hbm,
                         "frac": algo / (avg * 1e-3) / 1e9 / hbm,
                         "peak_source": "%s copy bandwidth" % src}}


def _single_configs(fw):
    """(name, n, dtype, edge p, BS (0: automatic), generator arguments, seed,
    with predecessors) of the single-graph workloads besides the headline."""
    return [("n1024_i32_bs32", 1024, fw.FW_I32, 1.0, 32, dict(lo=1, hi=100), 1, True),
            ("n8192_i32_p0.5", 8192, fw.FW_I32, 0.5, 0, dict(lo=1, hi=1000), 2, True),
            ("n8192_f32_p0.5", 8192, fw.FW_F32, 0.5, 0, dict(kind=0), 2, True),
            ("n8192_f32_p0.5_distance_only", 8192, fw.FW_F32, 0.5, 0, dict(kind=0), 2, False),
            ("n8192_f64_p0.5", 8192, fw.FW_F64, 0.5, 0, dict(kind=0), 2, True),
            ("n8192_i64_p0.5", 8192, fw.FW_I64, 0.5, 0, dict(lo=1, hi=10 ** 12), 2, True)]


def _torch_dtype(fw, dt):
    import torch
    return {fw.FW_I32: torch.int32, fw.FW_F32: torch.float32, fw.FW_I64: torch.int64,
            fw.FW_F64: torch.float64}[dt]


def _fill(fw, dt):
    import graphgen.device as gdev
    return {fw.FW_I32: gdev.fill_i32, fw.FW_F32: gdev.fill_f32, fw.FW_I64: gdev.fill_i64,
            fw.FW_F64: gdev.fill_f64}[dt]


def trace_config(fw, name, out_path):
    """One traced solve (every task) of a single-graph workload of bench_configs:
    writes tracing.summarize and tracing.critical_path as JSON."""
    import torch
    import graphgen.device as gdev
    from paper_2403_18619_gb300 import tracing
    spec = {c[0]: c for c in _single_configs(fw)}.get(name)
    if spec is None:
        raise SystemExit("unknown config %r" % name)
    _, n, dt, p, bs, gen, seed, with_pred = spec
    ld = fw.padded(n)
    W = torch.empty((n, ld), dtype=_torch_dtype(fw, dt), device="cuda")
    _fill(fw, dt)(W[:, :n], seed=seed, p=p, **gen)
    D = torch.empty_like(W)
    P = torch.empty((n, ld), dtype=torch.int32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    plan = fw.fw_solve_plan(n, fw.Options.default(bs=bs), sms, dtype=dt)
    R, look = plan["rounds"], plan["lookahead"]
    tr = torch.zeros((R ** 3, 10), dtype=torch.int64, device="cuda")
    opt = fw.Options.default(bs=bs, trace=tr.data_ptr(), trace_cap=R ** 3, trace_stride=1)
    for _ in range(3):  # the last solve is the one kept (warm)
        D.copy_(W)
        tr.zero_()
        fw.fw_solve_ex(D[:, :n], P[:, :n] if with_pred else None, opt)
        fw.fw_sync_status()
    t = tr.cpu().numpy()
    out = {"config": name, "n": n, "bs": plan["bs"], "rounds": R, "lookahead": look,
           "summary": tracing.summarize(t),
           "critical_path": tracing.critical_path(t, fw.fw_queue_tasks(R, look))}
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({"trace": out_path, "round_us": out["critical_path"].get("round_us")}),
          flush=True)


def bench_configs(fw, args, only=None):
    """The other single-graph workloads: n = 1024 complete digraph, int32
    U[1,100], BS = 32 (launch / latency-bound), and n = 8192, p = 0.5, as fp32
    (0,1] (with and without predecessors), int32 U[1,1000], fp64 (0,1] and
    int64 U[1,1e12], each against its own measured peak (fw_peak_probe of its
    dtype)."""
    import torch
    import graphgen.device as gdev
    out = {}
    peaks = {}
    for name, n, dt, p, bs, gen, seed, with_pred in _single_configs(fw):
        if only is not None and name != only:
            continue
        if dt not in peaks:
            peaks[dt] = fw.fw_peak_probe(dt)[0]
        ld = fw.padded(n)
        W = torch.empty((n, ld), dtype=_torch_dtype(fw, dt), device="cuda")
        _fill(fw, dt)(W[:, :n], seed=seed, p=p, **gen)
        D = torch.empty_like(W)
        P = torch.empty((n, ld), dtype=torch.int32, device="cuda")
        opt = fw.Options.default(bs=bs)
        # the fp64 solve runs on GB300's narrow FP64 pipe (about 1 s at n = 8192)
        steps = 3 if dt == fw.FW_F64 else max(3, args.steps)
        ts = []
        for i in range(2 + steps):
            D.copy_(W)
            a, b = _events(2)
            a.record()
            fw.fw_solve_ex(D[:, :n], P[:, :n] if with_pred else None, opt)
            b.record()
            fw.fw_sync_status()
            if i >= 2:
                ts.append(a.elapsed_time(b))
        t = sorted(ts)[len(ts) // 2]
        rps = n ** 3 / (t * 1e-3)
        out[name] = {"ms_median": t, "relax_per_s": rps, "frac_of_peak": rps / peaks[dt],
                     "peak_relax_per_s": peaks[dt], "steps": steps}
        del W, D, P
    return out


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import graphgen.device as gdev
    import paper_2403_18619_gb300 as fw

    n = args.n
    ld = fw.padded(n)
    stream = torch.cuda.current_stream()
    W = torch.empty((n, ld), dtype=torch.int32, device="cuda")
    gdev.fill_i32(W[:, :n], seed=SEED + rank, p=P_EDGE, lo=LO, hi=HI)
    D = torch.empty_like(W)
    P = torch.empty((n, ld), dtype=torch.int32, device="cuda")

    rps, per_clk, probe_mhz = fw.fw_peak_probe(fw.FW_I32)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    for e in ev0 + ev1 + k0 + k1:      # create the underlying CUDA events now
        e.record(stream)
    torch.cuda.synchronize()

    def step(i=None):
        D.copy_(W)
        if i is None:
            opt = fw.Options.default(bs=args.bs, driver=args.driver)
            fw.fw_solve_ex(D[:, :n], P[:, :n], opt, stream)
            return
        opt = fw.Options.default(bs=args.bs, driver=args.driver,
                                 ev_start=k0[i].cuda_event, ev_stop=k1[i].cuda_event)
        ev0[i].record(stream)
        fw.fw_solve_ex(D[:, :n], P[:, :n], opt, stream)
        ev1[i].record(stream)

    for _ in range(args.warmup):
        step()
    fw.fw_sync_status()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            step(i)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    fw.fw_sync_status()
    if world > 1:
        dist.barrier()
    step_ms = [ev0[i].elapsed_time(ev1[i]) for i in range(args.steps)]
    kern_ms = [k0[i].elapsed_time(k1[i]) for i in range(args.steps)]
    t_ms = reduce_max(sum(step_ms), world)
    relax = float(n) ** 3
    value = whole_job_rate(relax * args.steps, world, t_ms * 1e-3)

    # end to end through the host-buffer entry point (pinned memory, copies timed)
    e2e = None
    if args.e2e_steps > 0:
        Wh = torch.empty((n, ld), dtype=torch.int32, pin_memory=True)
        Wh.copy_(W.cpu())
        Dh = torch.empty_like(Wh).pin_memory()
        Ph = torch.empty_like(Wh).pin_memory()
        opt = fw.Options.default(bs=args.bs, driver=args.driver)
        times = []
        for i in range(args.e2e_steps + 1):
            # weights in, distances and predecessors out, each in its own
            # pinned buffer (the weights stay as they are for the next step)
            t0 = time.perf_counter()
            fw.fw_solve_host_io(Wh[:, :n], Dh[:, :n], Ph[:, :n], opt, stream)
            dt = time.perf_counter() - t0
            if i > 0:
                times.append(dt)
        te = reduce_max(sum(times) / len(times), world)
        e2e = {"value": whole_job_rate(relax, world, te), "unit": "relax/s",
               "h2d_bytes_per_step": n * ld * 4, "d2h_bytes_per_step": 2 * n * ld * 4,
               "ms_per_step": te * 1e3, "ms_each": [t * 1e3 for t in times],
               "api": "fw_solve_host_io (pinned host buffers)"}

    if rank != 0:
        return 0
    kern_avg_s = sum(kern_ms) / len(kern_ms) * 1e-3
    achieved = relax / kern_avg_s
    line = {
        "metric": "relaxations/s (n^3/t)",
        "value": value,
        "unit": "relax/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": workload_name(n), "n": n, "seed": SEED, "edge_p": P_EDGE, "weights": [LO, HI],
                   "bs": args.bs, "driver": "phased" if args.driver == 2 else "persistent",
                   "parallelism": "replicas x%d" % world,
                   "l2": "no flush: %.1f GiB of dist+pred per step, far above the 129 MB L2"
                         % (2.0 * n * n * 4 / 2 ** 30)},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": rps / 1e12,
                     "unit": "Trelax/s", "frac": achieved / rps,
                     "traffic": TRAFFIC_BYTES.get((n, args.bs, args.driver)),
                     "traffic_source": TRAFFIC_NOTE.get((n, args.bs, args.driver)),
                     "kernel": "k_persistent_ws<int,128>",
                     "peak_source": "fw_peak_probe (__viaddmin_u32 chains on all SMs, same "
                                    "process, %.1f relax/SM-clk at %.0f MHz)" % (per_clk,
                                                                                  probe_mhz)},
        "clocks": clocks.summary(),
        "gpu_launches": 3 * args.steps,  # init, persistent solver, predecessor resolution
        "wall_s_timed_region": wall,
        "step_ms_stats": step_stats(step_ms),
    }
    if e2e:
        line["e2e"] = e2e
    if not args.no_extras and world == 1:
        line["batched"] = bench_batched(fw, args)
        line["backward"] = bench_backward(fw, args)
        line["intermediate"] = bench_intermediate(fw, args)
        line["configs"] = bench_configs(fw, args)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--bs", type=int, default=BS)
    ap.add_argument("--driver", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and backward measurements")
    ap.add_argument("--config", default=None,
                    help="time only this one of the other workloads (n1024_i32_bs32, "
                         "n8192_i32_p0.5, n8192_f32_p0.5, n8192_f32_p0.5_distance_only, "
                         "n8192_f64_p0.5, n8192_i64_p0.5, backward, batched, intermediate) and "
                         "print its "
                         "result, e.g. to profile it")
    ap.add_argument("--trace-config", nargs=2, default=None, metavar=("NAME", "OUT.json"),
                    help="trace one solve of a single-graph workload (as --config) and write "
                         "the trace summary and its per-round critical path")
    ap.add_argument("--trace-batched", default=None, metavar="OUT.json",
                    help="trace one batched solve of the 512-graph workload and write its "
                         "summary by size class (no timing line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.trace_config:
        import torch
        import paper_2403_18619_gb300 as fw
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        trace_config(fw, args.trace_config[0], args.trace_config[1])
        return 0
    if args.trace_batched:
        import torch
        import paper_2403_18619_gb300 as fw
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        trace_batched(fw, args.trace_batched)
        return 0
    if args.config:
        import torch
        import paper_2403_18619_gb300 as fw
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        extra = {"backward": bench_backward, "batched": bench_batched,
                 "intermediate": bench_intermediate}
        if args.config in extra:
            fn = extra[args.config]
            print(json.dumps({"config": args.config, **fn(fw, args)}), flush=True)
            return 0
        res = bench_configs(fw, args, only=args.config)
        if not res:
            raise SystemExit("unknown --config %r" % args.config)
        print(json.dumps({"config": args.config, **res[args.config]}), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
