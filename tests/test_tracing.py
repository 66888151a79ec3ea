"""The task-trace decoder on a hand-built trace (no GPU)."""
import numpy as np
import pytest

from paper_2403_18619_gb300 import tracing


def _row(task, typ, sm, claimed, ready, issued, start, end, published, c7=0, c8=0):
    return [task | (typ << 32), sm, claimed, ready, issued, published, start, c7, c8, end]


def _trace():
    rows = [
        # pivot on SM 0: waits 2 us for its tile, computes 10 us
        _row(0, 0, 0, 1000, 3000, 3000, 3500, 13500, 14000,
             c7=100 | (900 << 32), c8=1000 | (1200 << 32)),
        # remaining tile on SM 1: 5 us compute
        _row(7, 3, 1, 1000, 1500, 1600, 2000, 7000, 7500,
             c7=30 | (40 << 20) | (5 << 40), c8=9000 | (10000 << 32)),
        # a second remaining tile on SM 1, 1 us after the first
        _row(8, 3, 1, 6000, 6500, 6600, 8000, 12000, 12500,
             c7=10 | (20 << 20) | (0 << 40), c8=8000 | (9000 << 32)),
    ]
    t = np.zeros((6, 10), np.uint64)   # cap above the tasks written: zero rows are skipped
    t[:3] = np.array(rows, dtype=np.uint64)
    return t


def test_decode_fields():
    d = tracing.decode(_trace())
    assert d["task"].tolist() == [0, 7, 8]
    assert d["type"].tolist() == [0, 3, 3]
    assert d["sm"].tolist() == [0, 1, 1]
    assert d["tile_wait"].tolist()[1:] == [30, 10]
    assert d["chunk_wait"].tolist()[1:] == [40, 20]
    assert d["pred_wait"].tolist()[1:] == [5, 0]
    assert d["relax_end"].tolist()[1:] == [9000, 8000]
    assert d["whole"].tolist() == [1200, 10000, 9000]
    assert d["loaded"][0] == 100 and d["relaxed"][0] == 900 and d["stored"][0] == 1000


def test_summary():
    s = tracing.summarize(_trace())
    assert s["tasks"] == 3
    assert s["span_us"] == pytest.approx((14000 - 1000) / 1e3)
    piv = s["types"]["pivot"]
    assert piv["compute_us"]["mean"] == pytest.approx(10.0)
    assert piv["input_wait_us"]["mean"] == pytest.approx(2.0)
    assert piv["publish_lag_us"]["mean"] == pytest.approx(0.5)
    assert piv["cycles"] == {"loads": 100.0, "relax": 800.0, "post": 100.0, "store_end": 200.0,
                             "whole": 1200.0}
    rem = s["types"]["remaining"]
    assert rem["compute_us"]["n"] == 2 and rem["compute_us"]["mean"] == pytest.approx(4.5)
    assert rem["cycles"]["relax"] == pytest.approx(((9000 - 70) + (8000 - 30)) / 2)
    assert rem["cycles"]["epilogue"] == pytest.approx(((10000 - 9000 - 5) + (9000 - 8000)) / 2)
    # SM 0 busy 10 us of 13, SM 1 busy 9 us of 13; one gap of 1 us on SM 1
    assert s["busy_fraction"]["sms"] == 2
    assert s["busy_fraction"]["min"] == pytest.approx(9 / 13)
    assert s["busy_fraction"]["mean"] == pytest.approx((10 / 13 + 9 / 13) / 2)
    assert s["gap_us"]["n"] == 1 and s["gap_us"]["mean"] == pytest.approx(1.0)


def test_empty_and_bad_shapes():
    assert tracing.summarize(np.zeros((4, 10), np.uint64)) == {"tasks": 0}
    with pytest.raises(ValueError):
        tracing.decode(np.zeros((4, 9), np.uint64))


def test_summarize_batched_by_size_class():
    """Graph ids in bits 40-63 of word 0; tasks grouped by the size class of
    their graph: graph 0 (n = 100, class n <= 128) has the pivot, graph 1
    (n = 700, class n <= 1024) the two remaining tiles."""
    t = _trace()
    t[1, 0] |= np.uint64(1) << np.uint64(40)
    t[2, 0] |= np.uint64(1) << np.uint64(40)
    d = tracing.decode(t)
    assert d["graph"].tolist() == [0, 1, 1] and d["type"].tolist() == [0, 3, 3]
    s = tracing.summarize_batched(t, ns=[100, 700], bs_per_graph=[32, 64])
    assert set(s["by_class"]) == {"n<=128", "n<=1024"}
    small, mid = s["by_class"]["n<=128"], s["by_class"]["n<=1024"]
    assert small["graphs"] == 1 and small["bs"] == [32] and small["pivot"]["tasks"] == 1
    assert small["pivot"]["compute_us"] == pytest.approx(10.0)
    assert small["pivot"]["input_wait_us"] == pytest.approx(2.0)
    assert mid["remaining"]["tasks"] == 2 and mid["remaining"]["compute_us"] == pytest.approx(4.5)
    # compute shares: pivot 10 us, tiles 5 + 4 us of 19 us
    assert small["compute_share"] == pytest.approx(10 / 19)
    assert s["compute_share_by_type"]["remaining"] == pytest.approx(9 / 19)
    assert mid["span_us"] == pytest.approx((12500 - 1000) / 1e3)


def test_critical_path_segments():
    """A two-round chain built by hand: pivot(0) -> panels (0,1), (1,0) ->
    remaining tile (1,1) of round 0 -> pivot(1); the segments are the gaps
    between the chain's timestamps."""
    # queue rows (type, round, ti, tj) of R = 2: task ids 0..7
    q = [(0, 0, 0, 0), (1, 0, 0, 1), (2, 0, 1, 0), (3, 0, 1, 1), (0, 1, 1, 1),
         (1, 1, 1, 0), (2, 1, 0, 1), (3, 1, 0, 0)]
    rows = [
        _row(0, 0, 0, 0, 0, 0, 1000, 3000, 3500),      # pivot: compute 2 us, publish 0.5
        _row(1, 1, 1, 0, 0, 0, 4000, 6000, 6200),      # row panel
        _row(2, 2, 2, 0, 0, 0, 4500, 7000, 7400),      # column panel (the later one)
        _row(3, 3, 3, 0, 0, 0, 8000, 9000, 9100),      # remaining tile (1,1)
        _row(4, 0, 4, 0, 0, 0, 10000, 12000, 12500),   # pivot(1)
    ]
    t = np.zeros((8, 10), np.uint64)
    t[:5] = np.array(rows, dtype=np.uint64)
    t[:5, 2] = 1   # claimed (non-zero rows are decoded)
    cp = tracing.critical_path(t, q)
    assert cp["rounds"] == 1
    s = cp["segments_us"]
    assert s["pivot"] == pytest.approx(2.0) and s["pivot_pub"] == pytest.approx(0.5)
    assert s["to_panels"] == pytest.approx(1.0)      # 3.5 -> 4.5 (the later start)
    assert s["panels"] == pytest.approx(2.5)         # 4.5 -> 7.0
    assert s["panel_pub"] == pytest.approx(0.4)
    assert s["to_tile"] == pytest.approx(0.6) and s["tile"] == pytest.approx(1.0)
    assert s["tile_pub"] == pytest.approx(0.1) and s["to_pivot"] == pytest.approx(0.9)
    assert cp["round_us"] == pytest.approx(9.0)      # 1.0 -> 10.0


def test_critical_path_fused_tile_and_pivot():
    """Rounds of a solve whose tile (r+1, r+1) carries the pivot of round r+1
    along (trace type 4, the pivot's own queue entry never traced): a round
    runs from one fused task to the next."""
    # queue rows of R = 3 (task ids by position); only the chain's tasks matter
    q = [(0, 0, 0, 0), (1, 0, 0, 1), (2, 0, 1, 0), (3, 0, 1, 1), (0, 1, 1, 1),
         (1, 1, 1, 2), (2, 1, 2, 1), (3, 1, 2, 2), (0, 2, 2, 2)]
    rows = [
        _row(3, 4, 0, 0, 0, 0, 1000, 4000, 4300),     # tile (1,1) of round 0 + pivot(1)
        _row(5, 1, 1, 0, 0, 0, 5000, 6000, 6100),     # row panel (1,2)
        _row(6, 2, 2, 0, 0, 0, 5200, 6500, 6800),     # column panel (2,1), the later one
        _row(7, 4, 3, 0, 0, 0, 7500, 9000, 9200),     # tile (2,2) of round 1 + pivot(2)
    ]
    t = np.zeros((9, 10), np.uint64)
    t[:4] = np.array(rows, dtype=np.uint64)
    t[:4, 2] = 1
    cp = tracing.critical_path(t, q)
    assert cp["fused"] and cp["rounds"] == 1
    s = cp["segments_us"]
    assert s["tile_pivot"] == pytest.approx(3.0) and s["pivot_pub"] == pytest.approx(0.3)
    assert s["to_panels"] == pytest.approx(0.9)       # 4.3 -> 5.2
    assert s["panels"] == pytest.approx(1.3)          # 5.2 -> 6.5
    assert s["panel_pub"] == pytest.approx(0.3) and s["to_tile"] == pytest.approx(0.7)
    assert cp["round_us"] == pytest.approx(6.5)       # 1.0 -> 7.5
    summary = tracing.summarize(t)
    assert "tile_pivot" in summary["types"]
