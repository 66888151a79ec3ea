"""GPU parity of the blocked FW solve (through the C ABI) against the CPU oracle.

int32: distances bit-exact, predecessors equal on every pair whose shortest
path is unique, and the shortest-path certificate on all the rest.
fp32: distances within 1e-6 * hops (relative) of the fp64 oracle, predecessors
equal where the oracle's last hop wins by a margin above that tolerance.
"""
import numpy as np
import pytest

import graphgen
import oracle
from fwtest import (INF, check_f32, check_f32_dist, check_int_full, check_int_rows, fw,
                    gpu_solve, gpu_solve_dist_only, int_case)

pytestmark = pytest.mark.gpu

PERSISTENT, PHASED = 1, 2


# ------------------------------------------------------------------ int32 ---

@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
@pytest.mark.parametrize("bs", [32, 64, 128])
@pytest.mark.parametrize("n", [1, 2, 5, 31, 33, 64, 130, 257, 600])
def test_int_sizes(n, bs, driver):
    W, Do, Po, cnt = int_case(n, 1000 + n, 0.35, 1, 60)
    D, P = gpu_solve(W, bs=bs, driver=driver)
    check_int_full(W, D, P, Do, Po, cnt)


@pytest.mark.parametrize("tile_tma", [0, 1])
@pytest.mark.parametrize("n,bs,extra_ld", [(33, 32, 0), (130, 64, 12), (257, 128, 4),
                                           (600, 128, 0)])
def test_tile_load_paths(n, bs, extra_ld, tile_tma):
    """The persistent driver's two ways of loading a remaining tile: one 2-D
    tensor copy (ragged edges zero-filled by the copy, masked by the kernel;
    padding columns never read) and one bulk copy per row."""
    W, Do, Po, cnt = int_case(n, 77 + n, 0.4, 1, 60)
    D, P = gpu_solve(W, bs=bs, driver=PERSISTENT, extra_ld=extra_ld, tile_tma=tile_tma)
    check_int_full(W, D, P, Do, Po, cnt)
    Wf = graphgen.dense_graph_f32(n, seed=n + 5, p=0.4)
    Dfo, Pfo = oracle.fw_f64(Wf)
    Df, Pf = gpu_solve(Wf, bs=bs, driver=PERSISTENT, extra_ld=extra_ld, tile_tma=tile_tma)
    check_f32(Wf, Df, Pf, Dfo, Pfo)


@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
def test_int_config_small(driver):
    """n=1024 complete digraph, weights uniform in [1,100], BS=32."""
    W, Do, Po, cnt = int_case(1024, 1, 1.0, 1, 100)
    D, P = gpu_solve(W, bs=32, driver=driver)
    check_int_full(W, D, P, Do, Po, cnt)


@pytest.mark.parametrize("bs", [32, 128])
def test_int_generic_path(bs):
    """Weights large enough that packed keys cannot hold the sums: every tile
    takes the generic kernel; also the packed path switched off by option."""
    n = 40
    W = graphgen.dense_graph_i32(n, seed=77, p=0.4, lo=1 << 20, hi=(1 << 23) + 5)
    Do, Po = oracle.fw_i64(W)
    cnt = oracle.path_count_i64(W, Do)
    for driver in (PERSISTENT, PHASED):
        D, P = gpu_solve(W, bs=bs, driver=driver)
        check_int_full(W, D, P, Do, Po, cnt)
    W2, Do2, Po2, cnt2 = int_case(300, 5, 0.3, 1, 50)
    D, P = gpu_solve(W2, bs=bs, packed=0)
    check_int_full(W2, D, P, Do2, Po2, cnt2)


def test_int_mixed_bounds():
    """Some tiles fit the packed keys and some do not, within one solve."""
    n = 300
    W = graphgen.dense_graph_i32(n, seed=8, p=0.5, lo=1, hi=40)
    big = graphgen.dense_graph_i32(n, seed=9, p=0.5, lo=1 << 19, hi=1 << 20)
    W[:, 200:] = np.where(W[:, 200:] < INF, big[:, 200:], INF)
    np.fill_diagonal(W, 0)
    Do, Po = oracle.fw_i64(W)
    cnt = oracle.path_count_i64(W, Do)
    D, P = gpu_solve(W, bs=32)
    check_int_full(W, D, P, Do, Po, cnt)


@pytest.mark.parametrize("bs", [32, 64, 128])
def test_int_key_only_snapshots(bs):
    """Panel values between a quarter of the packed-key cap and above it:
    panels whose values stay below the cap store their snapshot as keys only,
    and remaining tiles whose two panels' bounds add up beyond the cap decode
    those keys for the compare-and-select kernel; panels with larger values
    store raw snapshots too (every combination within one solve)."""
    n = 400
    cap = (1 << (31 - {32: 6, 64: 7, 128: 8}[bs])) - 1
    W = graphgen.dense_graph_i32(n, seed=bs, p=0.4, lo=1, hi=40)
    big = graphgen.dense_graph_i32(n, seed=bs + 1, p=0.4, lo=cap // 4, hi=cap // 2)
    W[:, 250:] = np.where(W[:, 250:] < INF, big[:, 250:], INF)
    W[300:, :] = np.where(W[300:, :] < INF, np.maximum(W[300:, :], cap // 3), INF)
    W[370:, :] = np.where(W[370:, :] < INF, cap + W[370:, :] % 1000, INF)
    np.fill_diagonal(W, 0)
    Do, Po = oracle.fw_i64(W)
    assert Do[Do < INF].max() > cap  # some values beyond the cap
    cnt = oracle.path_count_i64(W, Do)
    D, P = gpu_solve(W, bs=bs)
    check_int_full(W, D, P, Do, Po, cnt)


def test_int_padding_untouched_and_disconnected():
    n = 150
    W = graphgen.dense_graph_i32(n, seed=3, p=0.2, lo=1, hi=9)
    W[:70, 70:] = INF
    W[70:, :70] = INF
    np.fill_diagonal(W, 0)
    Do, Po = oracle.fw_i64(W)
    cnt = oracle.path_count_i64(W, Do)
    D, P = gpu_solve(W, bs=32, extra_ld=12)
    check_int_full(W, D, P, Do, Po, cnt)
    assert (D[:70, 70:] == INF).all() and (P[:70, 70:] == -1).all()


def test_int_zero_weight_edges():
    n = 90
    W = graphgen.dense_graph_i32(n, seed=12, p=0.3, lo=0, hi=5)
    Do, Po = oracle.fw_i64(W)
    D, P = gpu_solve(W, bs=32)
    np.testing.assert_array_equal(D.astype(np.int64), Do)
    # with zero weights pred may legitimately differ; it must still be a tight last hop
    cert = oracle.certificate_i64(W, D, P)
    assert cert[0] == 0 and cert[1] == 0 and cert[2] == 0


def test_task_trace_covers_every_task_in_order():
    """A traced persistent solve: one row per task, the queue's task mix, each
    task's timeline in causal order (claimed <= inputs ready <= compute start
    <= compute end <= published), and the solve itself still exact."""
    import torch
    from paper_2403_18619_gb300 import tracing
    m = fw()
    n, bs = 1000, 128
    R = (n + bs - 1) // bs
    W, Do, Po, cnt = int_case(n, 61, 0.5, 1, 90)
    tr = torch.zeros((R ** 3, 10), dtype=torch.int64, device="cuda")
    D = torch.from_numpy(W).cuda()
    P = torch.empty_like(D)
    opt = m.Options.default(bs=bs, driver=PERSISTENT, trace=tr.data_ptr(), trace_cap=R ** 3,
                            trace_stride=1)
    m.fw_solve_ex(D, P, opt)
    m.fw_sync_status()
    check_int_full(W, D.cpu().numpy(), P.cpu().numpy(), Do, Po, cnt)
    d = tracing.decode(tr.cpu().numpy())
    # every task of the queue but the pivots of rounds 1..R-1, which run
    # inside the task of tile (r, r) of round r-1 (trace type 4)
    q = m.fw_queue_tasks(R, m.fw_solve_plan(n, m.Options.default(bs=bs))["lookahead"])
    skipped = {k for k, (typ, r, i, j) in enumerate(q.tolist()) if typ == 0 and r >= 1}
    fused = {k for k, (typ, r, i, j) in enumerate(q.tolist())
             if typ == 3 and i == r + 1 and j == r + 1}
    assert sorted(d["task"].tolist()) == sorted(set(range(R ** 3)) - skipped)
    assert {t for t, ty in zip(d["task"].tolist(), d["type"].tolist()) if ty == 4} == fused
    counts = np.bincount(d["type"], minlength=5).tolist()
    assert counts == [1, R * (R - 1), R * (R - 1), R * (R - 1) ** 2 - (R - 1), R - 1]
    assert (d["claimed"] <= d["ready"]).all()
    assert (d["ready"] <= d["start"]).all()
    assert (d["start"] <= d["end"]).all()
    assert (d["end"] <= d["published"]).all()
    s = tracing.summarize(tr.cpu().numpy())
    assert s["tasks"] == R ** 3 - (R - 1) and 0 < s["busy_fraction"]["mean"] <= 1


def test_repeated_solves_share_workspace():
    cases = [int_case(n, 50 + n, 0.5, 1, 30) for n in (200, 520, 64)]
    for W, Do, Po, cnt in cases + cases[:1]:
        D, P = gpu_solve(W, bs=64)
        check_int_full(W, D, P, Do, Po, cnt)


def test_lookahead_and_grid_variants():
    W, Do, Po, cnt = int_case(700, 4, 0.6, 1, 80)
    for look, grid in ((0, 0), (1, 3), (10 ** 6, 0), (-1, 1)):
        D, P = gpu_solve(W, bs=32, lookahead=look, grid=grid)
        check_int_full(W, D, P, Do, Po, cnt)


def test_host_buffer_path():
    m = fw()
    W, Do, Po, cnt = int_case(333, 21, 0.4, 1, 99)
    ld = m.padded(333) + 4
    Dh = np.full((333, ld), -5, np.int32)
    Dh[:, :333] = W
    Ph = np.zeros((333, ld), np.int32)
    m.fw_solve_host(Dh[:, :333], Ph[:, :333], m.Options.default(bs=64))
    check_int_full(W, Dh[:, :333].copy(), Ph[:, :333].copy(), Do, Po, cnt)
    assert (Dh[:, 333:] == -5).all()


@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_host_buffer_path_events_and_repeats(dtype):
    """The host path with the caller's own start/stop events (the stop event
    also orders the early copy-back of the distances), on a non-default
    stream, solved twice into the same buffers."""
    import torch
    m = fw()
    n = 300
    if dtype == "i32":
        W, Do, Po, cnt = int_case(n, 8, 0.5, 1, 50)
    else:
        W = graphgen.dense_graph_f32(n, seed=8, p=0.5)
        Do, Po = oracle.fw_f64(W)
    s = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    e1.record(s)
    s.synchronize()
    for _ in range(2):
        Dh = np.array(W)
        Ph = np.full((n, n), 7, np.int32)
        opt = m.Options.default(bs=32, ev_start=e0.cuda_event, ev_stop=e1.cuda_event)
        m.fw_solve_host(Dh, Ph, opt, s)
        if dtype == "i32":
            check_int_full(W, Dh, Ph, Do, Po, cnt)
        else:
            check_f32(W, Dh, Ph, Do, Po)
        assert e0.elapsed_time(e1) > 0


@pytest.mark.parametrize("dtype", ["i32", "f64"])
def test_host_io_out_of_place(dtype):
    """fw_solve_host_io: the weights' host buffer is left unchanged, the
    results land in their own buffers (pinned tensors here, padded rows), and
    in place (dist is the weights' buffer) it is fw_solve_host."""
    import torch
    m = fw()
    n, ld = 301, 308
    if dtype == "i32":
        W, Do, Po, cnt = int_case(n, 9, 0.4, 1, 70)
    else:
        W = graphgen.dense_graph_f64(n, seed=9, p=0.4)
        Do, Po = oracle.fw_f64(W)
    tdt = torch.int32 if dtype == "i32" else torch.float64
    Wb = torch.zeros((n, ld), dtype=tdt, pin_memory=True)
    Wb[:, :n] = torch.from_numpy(W)
    Db = torch.full((n, ld), 5, dtype=tdt).pin_memory()
    Pb = torch.full((n, ld), 7, dtype=torch.int32).pin_memory()
    keep = Wb.clone()
    for _ in range(2):
        m.fw_solve_host_io(Wb[:, :n], Db[:, :n], Pb[:, :n])
        assert torch.equal(Wb, keep)                       # weights untouched, padding too
        assert (Db[:, n:] == 5).all() and (Pb[:, n:] == 7).all()
        D, P = Db[:, :n].numpy(), Pb[:, :n].numpy()
        if dtype == "i32":
            check_int_full(W, D, P, Do, Po, cnt)
        else:
            from test_gpu_wide import _check_f64
            _check_f64(W, D, P, Do, Po)
    # in place through the same entry point
    m.fw_solve_host_io(Wb[:, :n], Wb[:, :n], None)
    np.testing.assert_array_equal(Wb[:, :n].numpy(), Db[:, :n].numpy())
    with pytest.raises(ValueError):
        m.fw_solve_host_io(Wb[:, :n], Db[:, :n - 1], None)


# ------------------------------------------------------------------- fp32 ---

@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
@pytest.mark.parametrize("n,bs", [(37, 32), (200, 64), (513, 128), (1000, 64)])
def test_f32(n, bs, driver):
    W = graphgen.dense_graph_f32(n, seed=n, p=0.5)
    Do, Po = oracle.fw_f64(W)
    D, P = gpu_solve(W, bs=bs, driver=driver)
    safe = check_f32(W, D, P, Do, Po)
    assert safe > n


def test_f32_one_two_weights():
    n = 400
    W = graphgen.dense_graph_f32(n, seed=3, p=0.1, kind=graphgen.KIND_ONE_TWO)
    Do, Po = oracle.fw_f64(W)
    D, P = gpu_solve(W, bs=32)
    check_f32(W, D, P, Do, Po)


@pytest.mark.parametrize("n,bs", [(300, 32), (333, 64), (520, 128)])
def test_f32_integer_weights_exact(n, bs):
    """Integer-valued fp32 weights make every sum exact, with many equal-length
    paths.  Distances equal the int64 oracle's, predecessors equal it on unique
    paths and pass the shortest-path certificate everywhere (ties included),
    and the persistent and phased drivers (different task orders, snapshots
    and kernels for the remaining tiles) give bit-identical results: both
    keep the first step that reaches each minimum."""
    W = graphgen.dense_graph_i32(n, seed=n + 5, p=0.5, lo=1, hi=20)
    inf = graphgen.INF_I32
    Wf = np.where(W >= inf, np.inf, W).astype(np.float32)
    Do, Po = oracle.fw_i64(W)
    cnt = oracle.path_count_i64(W, Do)
    D, P = gpu_solve(Wf, bs=bs, driver=PERSISTENT)
    reach = np.isfinite(D)
    assert (reach == (Do < inf)).all(), "reachability differs"
    Di = np.where(reach, D, inf).astype(np.int32)
    check_int_full(W, Di, P, Do, Po, cnt)
    D2, P2 = gpu_solve(Wf, bs=bs, driver=PHASED)
    assert np.array_equal(D, D2, equal_nan=True)
    bad = np.argwhere(P != P2)
    assert len(bad) == 0, "drivers differ on %d predecessors, first %s: %d vs %d" % (
        len(bad), bad[0].tolist(), P[tuple(bad[0])], P2[tuple(bad[0])])


@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
def test_f32_argmin_every_step_improves(driver):
    """Entries that improve at every step of a 128-step block, in a row panel
    and in a remaining tile.  Vertex 0 reaches each k = 1..127 of block 0 at
    1000 - k, each of those k reaches every target 384..511 at 1, and the
    sources 256..383 reach each k of block 0 at 2000 - k.  In round 0 the row
    panel entry (0, j) improves at steps 1..127 (to 874) and the remaining
    tile entry (i, j) at every step 0..127 (2874 through vertex 0, then 2000 -
    k + 1): the strict minimum is the last step, k = 127.  This is the
    extreme case of the fp32 argmin accumulator (2^0 + ... + 2^127, which must
    stay below 2^128).  Distances and predecessors equal the int64 oracle's on
    every entry (all weights are integers, so every fp32 sum is exact)."""
    n, inf = 512, INF
    W = np.full((n, n), inf, np.int32)
    np.fill_diagonal(W, 0)
    k = np.arange(128)
    W[0, 1:128] = 1000 - k[1:]
    W[np.ix_(np.arange(256, 384), k)] = (2000 - k)[None, :]
    W[np.ix_(k[1:], np.arange(384, 512))] = 1
    Do, Po = oracle.fw_i64(W)
    cnt = oracle.path_count_i64(W, Do)
    assert Do[300, 400] == 1874 and Po[300, 400] == 127
    assert Do[0, 400] == 874 and Po[0, 400] == 127
    Wf = np.where(W >= inf, np.inf, W).astype(np.float32)
    D, P = gpu_solve(Wf, bs=128, driver=driver)
    reach = np.isfinite(D)
    assert (reach == (Do < inf)).all(), "reachability differs"
    check_int_full(W, np.where(reach, D, inf).astype(np.int32), P, Do, Po, cnt)
    assert (P[256:384, 384:] == 127).all() and (P[0, 384:] == 127).all()


# ---------------------------------------------------------- error paths ---

def test_negative_cycle_reported():
    import torch
    m = fw()
    n = 64
    W = graphgen.dense_graph_i32(n, seed=2, p=0.3, lo=1, hi=9)
    W[5, 6], W[6, 7], W[7, 5] = 1, 1, -10
    Wt = torch.from_numpy(W).cuda()
    with pytest.raises(m.FWError) as e:
        m.solve(Wt, m.Options.default(bs=32, packed_keys=0))
    assert e.value.code == 4
    Wf = torch.from_numpy(np.where(W >= INF, np.inf, W).astype(np.float32)).cuda()
    with pytest.raises(m.FWError) as e:
        m.solve(Wf, m.Options.default(bs=32))
    assert e.value.code == 4
    # the stream's status was cleared; a normal solve works afterwards
    Wg, Do, Po, cnt = int_case(100, 1, 0.5, 1, 10)
    D, P = gpu_solve(Wg, bs=32)
    check_int_full(Wg, D, P, Do, Po, cnt)


def test_dependency_timeout_is_reported_not_hung():
    """A task whose completion is never published: its dependents give up after
    the bounded wait and the host reads FW_ERR_TIMEOUT; the GPU stays usable."""
    import torch
    m = fw()
    n = 256
    W, Do, Po, cnt = int_case(n, 31, 0.5, 1, 50)
    R = n // 32
    q = m.fw_queue_tasks(R, 2 * 152)
    skip = int(np.argwhere(q[:, 0] == 1)[0][0])  # first row-panel task
    ld = m.padded(n)
    D = torch.from_numpy(W).cuda()
    P = torch.empty_like(D)
    opt = m.Options.default(bs=32, lookahead=2 * 152, debug_skip_release=skip,
                            timeout_ns=200_000_000)
    m.fw_solve_ex(D, P, opt)
    with pytest.raises(m.FWError) as e:
        m.fw_sync_status()
    assert e.value.code == 3
    D2, P2 = gpu_solve(W, bs=32)
    check_int_full(W, D2, P2, Do, Po, cnt)


# --------------------------------------------------------- verification ---

def test_certificate_kernel_matches_oracle():
    import torch
    m = fw()
    W, Do, Po, cnt = int_case(257, 17, 0.3, 1, 20)
    D, P = gpu_solve(W, bs=64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    assert m.fw_verify_certificate(t(W), t(D), t(P)).sum() == 0
    bad = D.copy()
    i, j = np.argwhere((Do > 0) & (Do < INF))[3]
    bad[i, j] += 1
    g = m.fw_verify_certificate(t(W), t(bad), t(P))
    c = oracle.certificate_i64(W, bad, P)
    assert g[0] == c[0] and g[1] + g[2] > 0 and c[1] + c[2] > 0
    badp = P.copy()
    badp[i, j] = (badp[i, j] + 1) % 257
    assert m.fw_verify_certificate(t(W), t(D), t(badp))[1] >= 1


def test_peak_probe_is_plausible():
    m = fw()
    for dt in (m.FW_I32, m.FW_F32):
        rps, per_clk, mhz = m.fw_peak_probe(dt)
        assert 8 <= per_clk <= 260, per_clk
        assert 300 <= mhz <= 2200, mhz
        assert rps > 1e12


def test_device_generator_matches_host():
    import torch
    import graphgen.device as gdev
    n = 777
    t = torch.empty((n, 780), dtype=torch.int32, device="cuda")
    gdev.fill_i32(t[:, :n], seed=5, p=0.3, lo=1, hi=1000)
    np.testing.assert_array_equal(t[:, :n].cpu().numpy(),
                                  graphgen.dense_graph_i32(n, 5, 0.3, 1, 1000))
    f = torch.empty((n, 780), dtype=torch.float32, device="cuda")
    gdev.fill_f32(f[:, :n], seed=6, p=0.5, kind=0)
    np.testing.assert_array_equal(f[:, :n].cpu().numpy(), graphgen.dense_graph_f32(n, 6, 0.5))
    gdev.fill_f32(f[:, :n], seed=6, p=0.5, kind=1)
    np.testing.assert_array_equal(f[:, :n].cpu().numpy(),
                                  graphgen.dense_graph_f32(n, 6, 0.5, kind=1))


# --------------------------------------------------------- distance only ---

@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
@pytest.mark.parametrize("n,bs,extra_ld", [(1, 32, 0), (33, 32, 4), (257, 128, 0), (600, 64, 8)])
def test_distance_only(n, bs, extra_ld, driver):
    """pred = NULL: the same distances (int32 bit-exact, fp32 within the
    tolerance), no predecessor work, padding untouched."""
    W, Do, Po, cnt = int_case(n, 300 + n, 0.4, 1, 60)
    D = gpu_solve_dist_only(W, bs=bs, driver=driver, extra_ld=extra_ld)
    np.testing.assert_array_equal(D.astype(np.int64), Do)
    Wf = graphgen.dense_graph_f32(n, seed=n + 11, p=0.4)
    Dfo, Pfo = oracle.fw_f64(Wf)
    Df = gpu_solve_dist_only(Wf, bs=bs, driver=driver, extra_ld=extra_ld)
    check_f32_dist(Wf, Df, Dfo, Pfo)


@pytest.mark.parametrize("packed", [0, 1])
def test_distance_only_generic_and_large_weights(packed):
    """Distance-only through the generic int32 kernels: large weights (beyond
    the packed-key bound) and the packed path switched off."""
    n = 300
    W = graphgen.dense_graph_i32(n, seed=41, p=0.3, lo=1 << 18, hi=1 << 19)
    Do, _ = oracle.fw_i64(W)
    D = gpu_solve_dist_only(W, bs=64, packed=packed)
    np.testing.assert_array_equal(D.astype(np.int64), Do)


def test_distance_only_host_and_noalloc():
    import torch
    m = fw()
    W, Do, Po, cnt = int_case(200, 9, 0.5, 1, 30)
    ld = m.padded(200)
    Dh = np.zeros((200, ld), np.int32)
    Dh[:, :200] = W
    m.fw_solve_host(Dh[:, :200], None)
    np.testing.assert_array_equal(Dh[:, :200].astype(np.int64), Do)
    D = torch.from_numpy(Dh.copy()).cuda()
    D[:, :200].copy_(torch.from_numpy(W))
    m.fw_solve_noalloc(D[:, :200], None)
    np.testing.assert_array_equal(D[:, :200].cpu().numpy().astype(np.int64), Do)
