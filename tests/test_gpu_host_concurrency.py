"""Host-side behaviour under concurrency and reuse: several host threads
solving on their own streams at once (each (device, stream) workspace has its
own lock), a batched plan fed alternating output buffers (its argument table
is refreshed on the stream; the recorded graph is reused), and the autograd
path's cached plans (a training step reuses the plan)."""
import threading

import numpy as np
import pytest

import graphgen
import oracle
from fwtest import fw

pytestmark = pytest.mark.gpu


def test_threads_on_their_own_streams():
    import torch
    m = fw()
    cases = [(300 + 37 * k, 60 + k) for k in range(6)]
    graphs = [graphgen.dense_graph_i32(n, seed=s, p=0.4, lo=1, hi=99) for n, s in cases]
    refs = [oracle.fw_i64(W)[0] for W in graphs]
    results, errors = [None] * len(cases), []

    def work(k):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for rep in range(3):
                    D, _ = m.solve(torch.from_numpy(graphs[k]).cuda(), stream=s)
                    results[k] = D.cpu().numpy()
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(120)
    assert not errors, errors
    for k in range(len(cases)):
        np.testing.assert_array_equal(results[k].astype(np.int64), refs[k])


def test_batched_plan_alternating_buffers():
    import torch
    m = fw()
    ns = [200, 333, 64, 500]
    lds = [m.padded(n) for n in ns]
    Ws = [graphgen.dense_graph_i32(n, seed=70 + i, p=0.3, lo=1, hi=50) for i, n in enumerate(ns)]
    refs = [oracle.fw_i64(W) for W in Ws]
    plan = m.BatchedPlan(ns, lds, m.FW_I32)
    sets = []
    for _ in range(2):
        D = [torch.empty((n, ld), dtype=torch.int32, device="cuda") for n, ld in zip(ns, lds)]
        P = [torch.empty((n, ld), dtype=torch.int32, device="cuda") for n, ld in zip(ns, lds)]
        sets.append((D, P))
    for rep in range(4):          # A, B, A, B: new buffers every call
        D, P = sets[rep % 2]
        for d, W, n in zip(D, Ws, ns):
            d[:, :n].copy_(torch.from_numpy(W))
            d[:, n:] = -1
        plan.solve([d[:, :n] for d, n in zip(D, ns)], [p[:, :n] for p, n in zip(P, ns)])
        m.fw_sync_status()
        for d, (Do, _), n in zip(D, refs, ns):
            np.testing.assert_array_equal(d[:, :n].cpu().numpy().astype(np.int64), Do)
            assert (d[:, n:] == -1).all()
    plan.close()


def test_autograd_reuses_its_batched_plan():
    import torch
    from paper_2403_18619_gb300 import autograd as ag
    ag.clear_plan_cache()
    B, n = 4, 96
    W = torch.from_numpy(np.stack([graphgen.dense_graph_f32(n, seed=80 + b, p=0.2,
                                                            kind=graphgen.KIND_ONE_TWO)
                                   for b in range(B)])).cuda()
    G = torch.from_numpy(graphgen.normal_f32((B, n, n), 3)).cuda()
    grads = []
    for step in range(3):
        Wt = W.clone().requires_grad_(True)
        D, _ = ag.shortest_paths(Wt)
        torch.autograd.backward(D.nan_to_num(posinf=0.0), grad_tensors=G)
        grads.append(Wt.grad.cpu().numpy())
        assert len(ag._PLANS) == 1          # one plan for (device, 4, 96, defaults)
    np.testing.assert_array_equal(grads[0], grads[1])
    np.testing.assert_array_equal(grads[0], grads[2])
    Do = np.stack([oracle.fw_f64(W[b].cpu().numpy())[0] for b in range(B)])
    Dg = ag.shortest_paths(W)[0].cpu().numpy()
    fin = np.isfinite(Do)
    assert (np.isfinite(Dg) == fin).all()
    assert (np.abs(Dg - Do)[fin] <= 1e-5 * np.abs(Do)[fin]).all()
    ag.clear_plan_cache()
    assert len(ag._PLANS) == 0
