"""Backward pass (dL/dW through the predecessor trees) against the fp64 oracle
gradient, central finite differences, and torch.autograd."""
import numpy as np
import pytest

import graphgen
import oracle
from fwtest import fw

pytestmark = pytest.mark.gpu


def _margin_instance(n, seed0, delta, p=0.3):
    # weights in [1, 2): w +- h (h = 2**-10) is exact in fp32 while w + h < 2
    for seed in range(seed0, seed0 + 2000):
        W = graphgen.dense_graph_f32(n, seed=seed, p=p, kind=graphgen.KIND_ONE_TWO)
        W = np.where(W >= 2 - 2 ** -9, np.float32(np.inf), W).astype(np.float32)
        np.fill_diagonal(W, 0)
        D, P = oracle.fw_f64(W)
        mg = oracle.lasthop_margin_f64(W, D, P)
        reach = np.isfinite(D) & ~np.eye(n, dtype=bool)
        if reach.sum() > n and (mg[reach] >= delta).all():
            return W, D, P
    pytest.skip("no instance with the required margin")


def _gpu_grad(W, G):
    import torch
    from paper_2403_18619_gb300.autograd import shortest_paths
    Wt = torch.from_numpy(W).cuda().requires_grad_(True)
    D, P = shortest_paths(Wt)
    L = (D.nan_to_num(posinf=0.0) * torch.from_numpy(G).cuda()).sum()
    L.backward()
    return Wt.grad.cpu().numpy().astype(np.float64), D.detach().cpu().numpy(), P.cpu().numpy()


@pytest.mark.parametrize("seed0", [300, 700])
def test_backward_vs_oracle_and_fd(seed0):
    n, h, delta = 32, 2.0 ** -10, 3 * 2.0 ** -10
    W, Do, Po = _margin_instance(n, seed0, delta)
    G = graphgen.adjoint_for(Do, seed=seed0 + 1).astype(np.float64)
    GW, D, P = _gpu_grad(W, G.astype(np.float32))
    reach = np.isfinite(Do) & ~np.eye(n, dtype=bool)
    np.testing.assert_array_equal(P[reach], Po[reach])
    GWo = oracle.grad_f64(G, Po)
    tol = 1e-5 * np.abs(GWo) + 1e-5 * np.linalg.norm(G)
    assert (np.abs(GW - GWo) <= tol).all()
    # central differences of the fp64 oracle on every edge
    edges = np.argwhere(np.isfinite(W) & ~np.eye(n, dtype=bool))
    fin = np.isfinite(Do)
    for (u, v) in edges[:: max(1, len(edges) // 60)]:
        Wp = W.copy(); Wp[u, v] += h
        Wm = W.copy(); Wm[u, v] -= h
        Dp, _ = oracle.fw_f64(Wp)
        Dm, _ = oracle.fw_f64(Wm)
        fd = (G[fin] * (Dp[fin] - Dm[fin])).sum() / (2 * h)
        assert abs(fd - GW[u, v]) <= 1e-5 * (1 + abs(fd)), (u, v, fd, GW[u, v])
    assert (GW[~np.isfinite(W)] == 0).all() and (np.diag(GW) == 0).all()


def test_backward_batched_config_shape():
    """64 graphs, n = 1024, p = 0.1, weights in [1, 2): one batched forward, one
    strided backward, through FWFunction.  The backward is a function of the
    predecessor trees, so EVERY row of EVERY graph is compared with the fp64
    oracle gradient through the GPU's own trees (no row filtered out).  The
    trees themselves are checked against the full fp64 oracle separately:
    each last hop equal to the oracle's or near-tight, distances within
    1e-6 * hops."""
    import torch
    from fwtest import check_pred_near_tight_f32
    from paper_2403_18619_gb300.autograd import shortest_paths
    B, n = 64, 1024
    Ws = np.stack([graphgen.dense_graph_f32(n, seed=500 + b, p=0.1, kind=graphgen.KIND_ONE_TWO)
                   for b in range(B)])
    Wt = torch.from_numpy(Ws).cuda().requires_grad_(True)
    D, P = shortest_paths(Wt)
    Dh = D.detach().cpu().numpy()
    Ph = P.cpu().numpy()
    Gs = np.stack([graphgen.adjoint_for(Dh[b], seed=900 + b) for b in range(B)])
    L = (D.nan_to_num(posinf=0.0) * torch.from_numpy(Gs).cuda()).sum()
    L.backward()
    GW = Wt.grad.cpu().numpy().astype(np.float64)
    differ = 0
    for b in range(B):
        # the forward's trees against the oracle's
        Do, Po = oracle.fw_f64(Ws[b])
        reach = np.isfinite(Do)
        assert (np.isfinite(Dh[b]) == reach).all(), b
        hops = oracle.hops(Po)
        tol = 1e-6 * np.maximum(hops, 1) * np.abs(Do)
        tol[~reach] = 0
        err = np.abs(Dh[b].astype(np.float64) - Do)
        err[~reach] = 0
        assert (err <= tol).all(), b
        differ += check_pred_near_tight_f32(Ws[b], Do, Ph[b], Po, tol)
        # the backward against the oracle gradient through the same trees
        G = Gs[b].astype(np.float64)
        GWo = oracle.grad_f64(G, Ph[b])
        gtol = 1e-5 * np.abs(GWo) + 1e-5 * np.linalg.norm(G)
        worst = np.max(np.abs(GW[b] - GWo) - gtol)
        assert worst <= 0, (b, worst)
        assert (GW[b][~np.isfinite(Ws[b])] == 0).all() and (np.diag(GW[b]) == 0).all()
    assert differ < 0.01 * B * n * n, differ


def test_backward_recompute_matches_stored():
    import torch
    from paper_2403_18619_gb300.autograd import shortest_paths
    n = 200
    W = graphgen.dense_graph_f32(n, seed=77, p=0.2, kind=graphgen.KIND_ONE_TWO)
    G = torch.from_numpy(graphgen.normal_f32((n, n), 5)).cuda()
    grads = []
    for rec in (False, True):
        Wt = torch.from_numpy(W).cuda().requires_grad_(True)
        D, _ = shortest_paths(Wt, recompute=rec)
        (D.nan_to_num(posinf=0.0) * G).sum().backward()
        grads.append(Wt.grad.cpu().numpy())
    np.testing.assert_array_equal(grads[0], grads[1])
