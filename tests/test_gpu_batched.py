"""Batched solve (many graphs of uneven size in one persistent launch) against
the CPU oracle, graph by graph, through the C ABI."""
import numpy as np
import pytest

import graphgen
import oracle
from fwtest import INF, check_f32, check_f32_dist, check_int_full, fw

pytestmark = pytest.mark.gpu


def _run(Ws, options=None, reps=1, with_pred=True):
    import torch
    m = fw()
    Ds, Ps, ns, lds = [], [], [], []
    for W in Ws:
        n = W.shape[0]
        ld = m.padded(n) + 4
        tdt = torch.int32 if W.dtype == np.int32 else torch.float32
        Db = torch.full((n, ld), -7, dtype=tdt, device="cuda")
        Pb = torch.full((n, ld), -9, dtype=torch.int32, device="cuda")
        Ds.append(Db)
        Ps.append(Pb)
        ns.append(n)
        lds.append(ld)
    plan = m.BatchedPlan(ns, lds, m.FW_I32 if Ws[0].dtype == np.int32 else m.FW_F32, options)
    for _ in range(reps):
        for W, Db in zip(Ws, Ds):
            Db[:, :W.shape[0]].copy_(torch.from_numpy(W))
        plan.solve([D[:, :n] for D, n in zip(Ds, ns)],
                   [P[:, :n] for P, n in zip(Ps, ns)] if with_pred else None)
        m.fw_sync_status()
    bs, tasks = plan.info()
    plan.close()
    out = []
    for D, P, n in zip(Ds, Ps, ns):
        Dh, Ph = D.cpu().numpy(), P.cpu().numpy()
        assert (Dh[:, n:] == -7).all() and (Ph[:, n:] == -9).all(), "padding written"
        out.append((Dh[:, :n].copy(), Ph[:, :n].copy()))
    return out, bs, tasks


def _int_batch(seed, count, lo_n, hi_n, p=0.3, whi=100):
    ns = graphgen.batch_sizes(seed, count, lo_n, hi_n)
    return [graphgen.dense_graph_i32(int(n), seed=seed * 1000 + b, p=p, lo=1, hi=whi)
            for b, n in enumerate(ns)]


@pytest.mark.parametrize("bs", [0, 32, 64, 128])
def test_batched_int_mixed_sizes(bs):
    Ws = _int_batch(3, 24, 1, 300)
    m = fw()
    out, bsv, tasks = _run(Ws, m.Options.default(bs=bs))
    if bs:
        assert (bsv == bs).all()
    for W, (D, P) in zip(Ws, out):
        Do, Po = oracle.fw_i64(W)
        check_int_full(W, D, P, Do, Po, oracle.path_count_i64(W, Do))


@pytest.mark.parametrize("seed", [3, 11])
def test_batched_shuffled_claim_order(seed):
    """The debug shuffle claims every wave segment's tasks in a random order
    (int32 and fp32 graphs of mixed sizes and block sizes): the dependency
    flags alone keep the results equal to the oracle's."""
    m = fw()
    Ws = _int_batch(20 + seed, 16, 20, 700, p=0.4)
    out, _, _ = _run(Ws, m.Options.default(debug_shuffle=seed))
    for W, (D, P) in zip(Ws, out):
        Do, Po = oracle.fw_i64(W)
        check_int_full(W, D, P, Do, Po, oracle.path_count_i64(W, Do))
    ns = graphgen.batch_sizes(30 + seed, 8, 20, 400)
    Wf = [graphgen.dense_graph_f32(int(n), seed=300 + b, p=0.5) for b, n in enumerate(ns)]
    out, _, _ = _run(Wf, m.Options.default(debug_shuffle=seed))
    for W, (D, P) in zip(Wf, out):
        Do, Po = oracle.fw_f64(W)
        check_f32(W, D, P, Do, Po)


def test_batched_replay_and_new_buffers():
    Ws = _int_batch(5, 12, 30, 200, p=0.5)
    out, _, _ = _run(Ws, reps=3)          # recorded once, replayed twice
    for W, (D, P) in zip(Ws, out):
        Do, Po = oracle.fw_i64(W)
        check_int_full(W, D, P, Do, Po, oracle.path_count_i64(W, Do))


def test_batched_generic_path_and_fp32():
    Ws = _int_batch(7, 8, 20, 140, p=0.4, whi=(1 << 22))
    out, _, _ = _run(Ws)
    for W, (D, P) in zip(Ws, out):
        Do, Po = oracle.fw_i64(W)
        check_int_full(W, D, P, Do, Po, oracle.path_count_i64(W, Do))
    ns = graphgen.batch_sizes(9, 10, 10, 260)
    Wf = [graphgen.dense_graph_f32(int(n), seed=90 + b, p=0.5) for b, n in enumerate(ns)]
    out, _, _ = _run(Wf)
    for W, (D, P) in zip(Wf, out):
        Do, Po = oracle.fw_f64(W)
        check_f32(W, D, P, Do, Po)


def test_batched_config_shape_sampled():
    """The 512-graph workload (n uniform in [64, 2048], p = 0.3, weights in
    [1, 100]): every graph checked by the GPU certificate, a sample of graphs
    against the full oracle."""
    import torch
    m = fw()
    ns = graphgen.batch_sizes(11, 512, 64, 2048)
    Ws = [graphgen.dense_graph_i32(int(n), seed=11000 + b, p=0.3, lo=1, hi=100)
          for b, n in enumerate(ns)]
    out, bsv, tasks = _run(Ws)
    assert tasks > 0
    for b in range(len(Ws)):
        W, (D, P) = Ws[b], out[b]
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        bad = m.fw_verify_certificate(t(W), t(D), t(P))
        assert bad.sum() == 0, (b, bad.tolist())
    rng = np.random.default_rng(0)
    for b in rng.choice(len(Ws), 5, replace=False):
        W, (D, P) = Ws[b], out[b]
        Do, Po = oracle.fw_i64(W)
        check_int_full(W, D, P, Do, Po, oracle.path_count_i64(W, Do))


def test_bs_table_and_autotune():
    """The autotuner fills the table of the element type it measured, for the
    classes up to max_n, and leaves the other type's table alone."""
    m = fw()
    old_i, old_f = m.fw_bs_table(), m.fw_bs_table(dtype=m.FW_F32)
    try:
        for dt, other in ((m.FW_I32, m.FW_F32), (m.FW_F32, m.FW_I32)):
            before = m.fw_bs_table(dtype=other)
            table, ms = m.fw_autotune_bs(dt, graphs_per_class=6, max_n=300)
            assert set(table.tolist()) <= {32, 64, 128}
            assert (ms[:3] > 0).all() and (ms[3:] == 0).all()
            assert (m.fw_bs_table(dtype=dt) == table).all()
            assert (m.fw_bs_table(dtype=other) == before).all()
    finally:
        m.fw_bs_table(old_i)
        m.fw_bs_table(old_f, dtype=m.FW_F32)


def test_batched_distance_only():
    """preds = NULL: every graph solved for distances only (int32 exact, fp32
    within tolerance); the predecessor buffers are never written."""
    Ws = _int_batch(21, 20, 1, 400)
    out, _, _ = _run(Ws, with_pred=False)
    for W, (D, P) in zip(Ws, out):
        Do, _ = oracle.fw_i64(W)
        np.testing.assert_array_equal(D.astype(np.int64), Do)
        assert (P == -9).all(), "pred written by a distance-only solve"
    ns = graphgen.batch_sizes(22, 8, 1, 300)
    Wf = [graphgen.dense_graph_f32(int(n), seed=2200 + b, p=0.3) for b, n in enumerate(ns)]
    out, _, _ = _run(Wf, with_pred=False)
    for W, (D, P) in zip(Wf, out):
        Do, Po = oracle.fw_f64(W)
        check_f32_dist(W, D, Do, Po)
