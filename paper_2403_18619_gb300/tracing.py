"""Decoder of the persistent driver's per-task trace (``fw_options.trace``).

The trace is the GPU view of the idle time that the paper's Opt-9 variants
remove (Sec. 3.2, measured in Sec. 4.3): for every sampled task, when it was
claimed, when its inputs were ready, when its operands were issued, when the
compute warps started and finished it, and when it was published.  The buffer
(``trace_cap`` rows of 10 uint64, filled on the device; include/fw.h) holds:

  [0] task index | type << 32   (0 pivot, 1 row panel, 2 column panel, 3 remaining tile)
  [1] SM id
  [2] claimed  [3] inputs ready  [4] operands issued  [5] published   (%globaltimer, ns)
  [6] compute start  [9] compute end                                  (%globaltimer, ns)
  [7] [8] SM-cycle counts of the task's phases:
      remaining tile: [7] = tile-load wait | chunk waits << 20 | predecessor-tile
                      wait << 40 (20 bits each), [8] = relaxation end | whole << 32
      pivot / panel:  [7] = operands loaded | relaxed << 32,
                      [8] = results stored | whole << 32

Rows that no task wrote (all zero) are skipped.  Pure numpy; no GPU needed.
"""
from __future__ import annotations

import numpy as np

TYPES = ("pivot", "row_panel", "col_panel", "remaining")


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
        if ty == 3:
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
