"""Decoder of the persistent driver's per-task trace (``fw_options.trace``).

The trace is the GPU view of the idle time that the paper's Opt-9 variants
remove (Sec. 3.2, measured in Sec. 4.3): for every sampled task, when it was
claimed, when its inputs were ready, when its operands were issued, when the
compute warps started and finished it, and when it was published.  The buffer
(``trace_cap`` rows of 10 uint64, filled on the device; include/fw.h) holds:

  [0] task index | type << 32 | graph << 40   (type: 0 pivot, 1 row panel,
      2 column panel, 3 remaining tile, 4 remaining tile (r+1, r+1) of round
      r followed on the same SM by the pivot of round r+1, whose own queue
      entry is then skipped; graph: the graph of a batched solve)
  [1] SM id
  [2] claimed  [3] inputs ready  [4] operands issued  [5] published   (%globaltimer, ns)
  [6] compute start  [9] compute end                                  (%globaltimer, ns)
  [7] [8] SM-cycle counts of the task's phases:
      remaining tile: [7] = tile-load wait | chunk waits << 20 | predecessor-tile
                      wait << 40 (20 bits each), [8] = relaxation end | whole << 32
                      (type 4: of its tile part)
      pivot / panel:  [7] = operands loaded | relaxed << 32,
                      [8] = results stored | whole << 32

Rows that no task wrote (all zero) are skipped.  Pure numpy; no GPU needed.
"""
from __future__ import annotations

import numpy as np

TYPES = ("pivot", "row_panel", "col_panel", "remaining", "tile_pivot")


def decode(trace) -> dict:
    """Columns of the written rows of a trace buffer (numpy or CPU tensor of
    shape (cap, 10)), as int64 arrays keyed by name."""
    t = np.asarray(trace).astype(np.uint64)
    if t.ndim != 2 or t.shape[1] != 10:
        raise ValueError("a trace buffer has 10 columns, got shape %s" % (t.shape,))
    t = t[t[:, 2] != 0]
    c7, c8 = t[:, 7], t[:, 8]
    m20, m32 = np.uint64(0xFFFFF), np.uint64(0xFFFFFFFF)
    return {
        "task": (t[:, 0] & m32).astype(np.int64),
        "type": ((t[:, 0] >> np.uint64(32)) & np.uint64(0xFF)).astype(np.int64),
        "graph": (t[:, 0] >> np.uint64(40)).astype(np.int64),
        "sm": t[:, 1].astype(np.int64),
        "claimed": t[:, 2].astype(np.int64),
        "ready": t[:, 3].astype(np.int64),
        "issued": t[:, 4].astype(np.int64),
        "published": t[:, 5].astype(np.int64),
        "start": t[:, 6].astype(np.int64),
        "end": t[:, 9].astype(np.int64),
        # remaining-tile phase cycles
        "tile_wait": (c7 & m20).astype(np.int64),
        "chunk_wait": ((c7 >> np.uint64(20)) & m20).astype(np.int64),
        "pred_wait": ((c7 >> np.uint64(40)) & m20).astype(np.int64),
        "relax_end": (c8 & m32).astype(np.int64),
        "whole": (c8 >> np.uint64(32)).astype(np.int64),
        # pivot / panel phase cycles (same words, other fields)
        "loaded": (c7 & m32).astype(np.int64),
        "relaxed": (c7 >> np.uint64(32)).astype(np.int64),
        "stored": (c8 & m32).astype(np.int64),
    }


def _stats(x) -> dict:
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return {"n": 0}
    return {"n": int(x.size), "mean": float(x.mean()), "p50": float(np.median(x)),
            "p99": float(np.percentile(x, 99)), "max": float(x.max())}


def summarize(trace) -> dict:
    """Per task type: compute time, wait for inputs (claim to ready) and
    publication lag (compute end to published), in microseconds; per SM: the
    compute warps' busy fraction of the traced span and the gaps between
    consecutive tasks; phase cycle means per task type.  With a trace stride
    above 1 the busy fractions and gaps cover the sampled tasks only."""
    d = decode(trace)
    out = {"tasks": int(d["task"].size)}
    if d["task"].size == 0:
        return out
    t0 = int(min(d["claimed"].min(), d["start"].min()))
    span = int(max(d["end"].max(), d["published"].max())) - t0
    out["span_us"] = span / 1e3
    comp = (d["end"] - d["start"]) / 1e3
    wait = (d["ready"] - d["claimed"]) / 1e3
    lag = (d["published"] - d["end"]) / 1e3
    per_type = {}
    for ty, name in enumerate(TYPES):
        m = d["type"] == ty
        if not m.any():
            continue
        e = {"compute_us": _stats(comp[m]), "input_wait_us": _stats(wait[m]),
             "publish_lag_us": _stats(lag[m])}
        if ty in (3, 4):
            relax = d["relax_end"][m] - d["tile_wait"][m] - d["chunk_wait"][m]
            e["cycles"] = {
                "tile_wait": float(d["tile_wait"][m].mean()),
                "chunk_wait": float(d["chunk_wait"][m].mean()),
                "relax": float(relax.mean()),
                "pred_wait": float(d["pred_wait"][m].mean()),
                "epilogue": float((d["whole"][m] - d["relax_end"][m] - d["pred_wait"][m]).mean()),
                "whole": float(d["whole"][m].mean()),
            }
        else:
            e["cycles"] = {
                "loads": float(d["loaded"][m].mean()),
                "relax": float((d["relaxed"][m] - d["loaded"][m]).mean()),
                "post": float((d["stored"][m] - d["relaxed"][m]).mean()),
                "store_end": float((d["whole"][m] - d["stored"][m]).mean()),
                "whole": float(d["whole"][m].mean()),
            }
        per_type[name] = e
    out["types"] = per_type
    busy, gaps = [], []
    for s in np.unique(d["sm"]):
        m = np.where(d["sm"] == s)[0]
        o = m[np.argsort(d["start"][m], kind="stable")]
        busy.append(float((d["end"][o] - d["start"][o]).sum()) / span if span > 0 else 0.0)
        gaps.append((d["start"][o][1:] - d["end"][o][:-1]) / 1e3)
    out["busy_fraction"] = {"mean": float(np.mean(busy)), "min": float(np.min(busy)),
                            "sms": len(busy)}
    out["gap_us"] = _stats(np.concatenate(gaps) if gaps else np.zeros(0))
    return out


def summarize_batched(trace, ns, bs_per_graph, bounds=(128, 256, 512, 1024, 2048)) -> dict:
    """A batched solve's trace by size class of the graphs (n <= bound): per
    class and task type the tasks, the mean compute time and the mean wait for
    inputs (claim to ready, microseconds), the class's share of the compute
    time, and the span from its first claim to its last publication; overall,
    the busy fraction of the compute warps and the share of compute time per
    task type.  ns, bs_per_graph: vertex count and block size of every graph."""
    d = decode(trace)
    out = summarize(trace)
    if d["task"].size == 0:
        return out
    ns = np.asarray(ns, np.int64)
    bsg = np.asarray(bs_per_graph, np.int64)
    cls = np.searchsorted(np.asarray(bounds), ns[d["graph"]], side="left")
    comp = (d["end"] - d["start"]).astype(np.float64) / 1e3
    wait = (d["ready"] - d["claimed"]).astype(np.float64) / 1e3
    total = comp.sum()
    out["compute_share_by_type"] = {TYPES[t]: float(comp[d["type"] == t].sum() / total)
                                    for t in range(len(TYPES)) if (d["type"] == t).any()}
    by = {}
    for c in np.unique(cls):
        m = cls == c
        name = "n<=%d" % bounds[c] if c < len(bounds) else "n>%d" % bounds[-1]
        g = np.unique(d["graph"][m])
        e = {"graphs": int(g.size), "bs": sorted(set(int(x) for x in bsg[g])),
             "compute_share": float(comp[m].sum() / total),
             "span_us": float((d["published"][m].max() - d["claimed"][m].min()) / 1e3)}
        for t in range(len(TYPES)):
            mt = m & (d["type"] == t)
            if mt.any():
                e[TYPES[t]] = {"tasks": int(mt.sum()), "compute_us": float(comp[mt].mean()),
                               "input_wait_us": float(wait[mt].mean())}
        by[name] = e
    out["by_class"] = by
    return out


CHAIN = ("pivot", "row_panel", "col_panel", "remaining")


def critical_path(trace, queue) -> dict:
    """Per-round breakdown of the chain that bounds a solve with few tiles:
    pivot(r) -> panels (r, r+1) and (r+1, r) -> remaining tile (r+1, r+1) of
    round r -> pivot(r+1) (Sec. 2.3: the next round's pivot tile is the last
    tile round r updates on its path).  queue: the solve's task list, one row
    (type, round, tile row, tile column) per task index (fw_queue_tasks).  For
    every round with all five tasks traced, the segments (microseconds, means
    over rounds):
      pivot      compute of pivot(r)      pivot_pub  its publication
      to_panels  publication to the later panel's compute start
      panels     the two panels' compute (to the later end)
      panel_pub  their publication
      to_tile    to the remaining tile's compute start
      tile       its compute          tile_pub   its publication
      to_pivot   to pivot(r+1)'s compute start
    and their sum, the round time along the chain.  When the engine fuses
    tile (r+1, r+1) with pivot(r+1) (trace type 4), a round r >= 1 runs from
    the fused task of round r-1 to that of round r:
      tile_pivot  compute of tile (r, r) of round r-1 and of pivot(r)
      pivot_pub, to_panels, panels, panel_pub  as above
      to_tile     to the next fused task's compute start"""
    d = decode(trace)
    q = np.asarray(queue)
    key = {(int(t), int(r), int(i), int(j)): k for k, (t, r, i, j) in enumerate(q)}
    row = {int(t): k for k, t in enumerate(d["task"])}

    def get(typ, r, i, j):
        k = key.get((typ, r, i, j))
        return row.get(k) if k is not None else None

    st, en, pb = d["start"], d["end"], d["published"]
    R = int(q[:, 1].max()) + 1 if len(q) else 0
    fused = bool((d["type"] == 4).any())
    if fused:
        names = ("tile_pivot", "pivot_pub", "to_panels", "panels", "panel_pub", "to_tile")
        segs = {k: [] for k in names}
        for r in range(1, R - 1):
            ids = [get(3, r - 1, r, r), get(1, r, r, r + 1), get(2, r, r + 1, r),
                   get(3, r, r + 1, r + 1)]
            if any(x is None for x in ids):
                continue
            fp, prow, pcol, nx = ids
            t = [st[fp], en[fp], pb[fp], max(st[prow], st[pcol]), max(en[prow], en[pcol]),
                 max(pb[prow], pb[pcol]), st[nx]]
            for k, a, b in zip(names, t[:-1], t[1:]):
                segs[k].append((b - a) / 1e3)
    else:
        names = ("pivot", "pivot_pub", "to_panels", "panels", "panel_pub", "to_tile", "tile",
                 "tile_pub", "to_pivot")
        segs = {k: [] for k in names}
        for r in range(R - 1):
            ids = [get(0, r, r, r), get(1, r, r, r + 1), get(2, r, r + 1, r),
                   get(3, r, r + 1, r + 1), get(0, r + 1, r + 1, r + 1)]
            if any(x is None for x in ids):
                continue
            pv, prow, pcol, tl, nx = ids
            t = [st[pv], en[pv], pb[pv], max(st[prow], st[pcol]), max(en[prow], en[pcol]),
                 max(pb[prow], pb[pcol]), st[tl], en[tl], pb[tl], st[nx]]
            for k, a, b in zip(names, t[:-1], t[1:]):
                segs[k].append((b - a) / 1e3)
    out = {"rounds": len(segs[names[0]]), "fused": fused}
    if out["rounds"]:
        means = {k: float(np.mean(v)) for k, v in segs.items()}
        out["segments_us"] = means
        out["round_us"] = float(sum(means.values()))
    return out
