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
    strided backward, checked against the fp64 oracle gradient on every source
    row whose tree matches the oracle's (the adjoint of other rows is zeroed on
    both sides)."""
    import torch
    from paper_2403_18619_gb300.autograd import shortest_paths
    B, n = 64, 1024
    Ws = np.stack([graphgen.dense_graph_f32(n, seed=500 + b, p=0.1, kind=graphgen.KIND_ONE_TWO)
                   for b in range(B)])
    Wt = torch.from_numpy(Ws).cuda().requires_grad_(True)
    D, P = shortest_paths(Wt)
    Ph = P.cpu().numpy()
    checked = 0
    Gs = np.zeros_like(Ws)
    oracle_grads = []
    for b in range(0, B, 16):
        Do, Po = oracle.fw_f64(Ws[b])
        G = graphgen.adjoint_for(Do, seed=900 + b).astype(np.float64)
        agree = (Ph[b] == Po).all(axis=1)
        G[~agree] = 0.0
        Gs[b] = G
        oracle_grads.append((b, oracle.grad_f64(G, Po), G))
        checked += agree.sum()
    L = (D.nan_to_num(posinf=0.0) * torch.from_numpy(Gs).cuda()).sum()
    L.backward()
    GW = Wt.grad.cpu().numpy().astype(np.float64)
    for b, GWo, G in oracle_grads:
        tol = 1e-5 * np.abs(GWo) + 1e-5 * np.linalg.norm(G)
        assert (np.abs(GW[b] - GWo) <= tol).all(), b
    assert checked > 0.9 * 4 * n
    # graphs given a zero adjoint get a zero gradient
    assert (GW[1] == 0).all()


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
