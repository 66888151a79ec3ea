"""Pins for the CPU oracle: it is checked against things other than itself.

* a hand-worked example (tests/golden/hand5.txt),
* closed forms (path graph, directed ring, unit-weight complete graph,
  disconnected graph),
* brute-force enumeration of every simple path (n <= 7),
* scipy's shortest_path / dijkstra (distances and last-hop predecessors),
* the triangle inequality and the certificate on its own output, plus planted
  faults that the certificate must catch,
* central finite differences for the gradient.

All of this runs on the CPU (no GPU marker).
"""
import itertools
import os

import numpy as np
import pytest

import graphgen
import oracle

INF = oracle.INF_I32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_hand5():
    lines = [l.split("#")[0].strip() for l in open(os.path.join(GOLDEN, "hand5.txt"))]
    lines = [l for l in lines if l]
    n = int(lines[0].split()[1])
    i = lines.index("edges") + 1
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    while lines[i] != "dist":
        u, v, w = map(int, lines[i].split())
        W[u, v] = w
        i += 1
    D = np.array([list(map(int, lines[i + 1 + r].split())) for r in range(n)], np.int64)
    j = lines.index("pred") + 1
    P = np.array([list(map(int, lines[j + r].split())) for r in range(n)], np.int32)
    return W, D, P


def brute_force(W, inf):
    """All simple paths: min distance and the set of last hops achieving it."""
    n = W.shape[0]
    best = np.full((n, n), np.inf)
    last = [[set() for _ in range(n)] for _ in range(n)]
    count = np.zeros((n, n), np.int64)
    for s in range(n):
        best[s, s] = 0
        others = [v for v in range(n) if v != s]
        for L in range(1, n):
            for mids in itertools.permutations(others, L - 1):
                for t in others:
                    if t in mids:
                        continue
                    path = (s,) + mids + (t,)
                    c = 0.0
                    ok = True
                    for a, b in zip(path[:-1], path[1:]):
                        w = W[a, b]
                        if (np.isinf(w) if W.dtype.kind == "f" else w >= inf):
                            ok = False
                            break
                        c += float(w)
                    if not ok:
                        continue
                    if c < best[s, t]:
                        best[s, t] = c
                        last[s][t] = {path[-2]}
                        count[s, t] = 1
                    elif c == best[s, t]:
                        last[s][t].add(path[-2])
                        count[s, t] += 1
    return best, last, count


def scipy_sp(W, method):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    Wf = W.astype(np.float64)
    if W.dtype.kind == "i":
        Wf[W >= INF] = np.inf
    G = sp.csgraph_from_dense(Wf, null_value=np.inf)
    return sp.shortest_path(G, method=method, directed=True, return_predecessors=True)


# ------------------------------------------------------------------ golden ---

def test_hand_example():
    W, D, P = load_hand5()
    Do, Po = oracle.fw_i64(W)
    np.testing.assert_array_equal(Do, D)
    np.testing.assert_array_equal(Po, P)
    Dd, Pd = oracle.dijkstra_i64(W, np.arange(5))
    np.testing.assert_array_equal(Dd, D)
    np.testing.assert_array_equal(Pd, P)


# ------------------------------------------------------------- closed forms ---

def test_path_graph():
    n = 9
    w = np.arange(1, n, dtype=np.int32) * 3
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    for k in range(n - 1):
        W[k, k + 1] = w[k]
    D, P = oracle.fw_i64(W)
    for i in range(n):
        for j in range(n):
            if i < j:
                assert D[i, j] == w[i:j].sum()
                assert P[i, j] == j - 1
            elif i > j:
                assert D[i, j] == INF and P[i, j] == -1
            else:
                assert D[i, j] == 0 and P[i, j] == -1


def test_directed_ring():
    n = 11
    w = (np.arange(n) % 4 + 1).astype(np.int32)
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    for k in range(n):
        W[k, (k + 1) % n] = w[k]
    D, P = oracle.fw_i64(W)
    for i in range(n):
        for j in range(n):
            steps = (j - i) % n
            assert D[i, j] == sum(w[(i + t) % n] for t in range(steps))
            assert P[i, j] == (-1 if i == j else (j - 1) % n)


def test_unit_complete_graph():
    n = 17
    W = np.ones((n, n), np.int32)
    np.fill_diagonal(W, 0)
    D, P = oracle.fw_i64(W)
    off = ~np.eye(n, dtype=bool)
    assert (D[off] == 1).all() and (np.diag(D) == 0).all()
    assert (P[off] == np.repeat(np.arange(n), n).reshape(n, n)[off]).all()
    Wf = W.astype(np.float32)
    Df, Pf = oracle.fw_f64(Wf)
    np.testing.assert_array_equal(Df, D.astype(np.float64))
    np.testing.assert_array_equal(Pf, P)


def test_disconnected():
    n = 12
    W = graphgen.dense_graph_i32(n, seed=5, p=1.0, lo=1, hi=9)
    W[:6, 6:] = INF
    W[6:, :6] = INF
    D, P = oracle.fw_i64(W)
    assert (D[:6, 6:] == INF).all() and (D[6:, :6] == INF).all()
    assert (P[:6, 6:] == -1).all() and (P[6:, :6] == -1).all()
    Da, _ = oracle.fw_i64(W[:6, :6])
    np.testing.assert_array_equal(D[:6, :6], Da)


# -------------------------------------------------------------- brute force ---

@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [5, 7])
def test_brute_force_int(seed, n):
    W = graphgen.dense_graph_i32(n, seed=seed, p=0.6, lo=1, hi=6)
    best, last, count = brute_force(W, INF)
    D, P = oracle.fw_i64(W)
    for s in range(n):
        for t in range(n):
            if np.isinf(best[s, t]):
                assert D[s, t] == INF and P[s, t] == -1
                continue
            assert D[s, t] == best[s, t]
            if s != t:
                assert P[s, t] in last[s][t]
                if count[s, t] == 1:
                    assert P[s, t] == next(iter(last[s][t]))
    cnt = oracle.path_count_i64(W, D)
    for s in range(n):
        for t in range(n):
            if s != t and not np.isinf(best[s, t]):
                assert cnt[s, t] == min(2, count[s, t])


@pytest.mark.parametrize("seed", [11, 12])
def test_brute_force_float(seed):
    n = 7
    W = graphgen.dense_graph_f32(n, seed=seed, p=0.7)
    best, last, count = brute_force(W, None)
    D, P = oracle.fw_f64(W)
    for s in range(n):
        for t in range(n):
            if np.isinf(best[s, t]):
                assert np.isinf(D[s, t]) and P[s, t] == -1
            else:
                assert abs(D[s, t] - best[s, t]) <= 1e-12 * max(1.0, best[s, t])
                if s != t and count[s, t] == 1:
                    assert P[s, t] in last[s][t]


# -------------------------------------------------------------- scipy pins ---

@pytest.mark.parametrize("n,p,seed", [(40, 0.3, 1), (97, 0.1, 2), (160, 0.5, 3)])
def test_vs_scipy_int(n, p, seed):
    W = graphgen.dense_graph_i32(n, seed=seed, p=p, lo=1, hi=50)
    D, P = oracle.fw_i64(W)
    dist, pred = scipy_sp(W, "FW")
    reach = np.isfinite(dist)
    assert ((D < INF) == reach).all()
    np.testing.assert_array_equal(D[reach], dist[reach].astype(np.int64))
    cnt = oracle.path_count_i64(W, D)
    uniq = (cnt == 1) & reach & ~np.eye(n, dtype=bool)
    ddist, dpred = scipy_sp(W, "D")
    np.testing.assert_array_equal(P[uniq], dpred[uniq])
    assert uniq.sum() > n  # the comparison is not vacuous
    Dd, Pd = oracle.dijkstra_i64(W, np.arange(n))
    np.testing.assert_array_equal(Dd, D)
    np.testing.assert_array_equal(Pd[uniq], P[uniq])


@pytest.mark.parametrize("n,p,seed", [(60, 0.3, 4), (128, 0.5, 5)])
def test_vs_scipy_float(n, p, seed):
    W = graphgen.dense_graph_f32(n, seed=seed, p=p)
    D, P = oracle.fw_f64(W)
    dist, pred = scipy_sp(W, "D")
    reach = np.isfinite(dist)
    assert (np.isfinite(D) == reach).all()
    np.testing.assert_allclose(D[reach], dist[reach], rtol=1e-12, atol=0)
    Dd, Pd = oracle.dijkstra_f64(W, np.arange(n))
    np.testing.assert_allclose(Dd[reach], D[reach], rtol=1e-12, atol=0)
    mg = oracle.lasthop_margin_f64(W, D, P)
    safe = reach & (mg > 1e-9 * np.maximum(D, 1))
    np.testing.assert_array_equal(P[safe], pred[safe])
    # the Dijkstra oracle's predecessors: scipy's on the same margin-safe pairs,
    # and a tight last hop (an edge whose use realises the distance) everywhere
    np.testing.assert_array_equal(Pd[safe], pred[safe])
    off = reach & ~np.eye(n, dtype=bool)
    i, j = np.nonzero(off)
    u = Pd[i, j]
    assert (u >= 0).all() and (u != j).all()
    Wd = W.astype(np.float64)
    assert np.isfinite(Wd[u, j]).all()
    np.testing.assert_allclose(Dd[i, u] + Wd[u, j], Dd[i, j], rtol=1e-12, atol=0)
    assert (Pd[~off] == -1).all()
    assert safe.sum() > n


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_wide_inputs(seed):
    """64-bit inputs: int64 weights far beyond the int32 range (every sum of up
    to 6 of them is exact in the brute force's fp64) and fp64 weights with full
    53-bit mantissas."""
    n = 7
    W = graphgen.dense_graph_i64(n, seed=seed, p=0.6, lo=1, hi=10 ** 12)
    best, last, count = brute_force(W, graphgen.INF_I64)
    D, P = oracle.fw_i64(W)
    for s_ in range(n):
        for t in range(n):
            if np.isinf(best[s_, t]):
                assert D[s_, t] == graphgen.INF_I64 and P[s_, t] == -1
                continue
            assert D[s_, t] == int(best[s_, t])
            if s_ != t:
                assert P[s_, t] in last[s_][t]
    V = graphgen.dense_graph_f64(n, seed=seed + 10, p=0.7)
    best, last, count = brute_force(V, None)
    D, P = oracle.fw_f64(V)
    for s_ in range(n):
        for t in range(n):
            if np.isinf(best[s_, t]):
                assert np.isinf(D[s_, t]) and P[s_, t] == -1
            else:
                assert abs(D[s_, t] - best[s_, t]) <= 1e-15 * 8 * max(1.0, best[s_, t])
                if s_ != t and count[s_, t] == 1:
                    assert P[s_, t] in last[s_][t]


def test_vs_scipy_wide_inputs():
    """int64 weights up to 1e12 (every path sum below 2**53, so scipy's fp64
    distances are exact) and fp64 weights: distances equal (int64) or within
    1e-13 relative (fp64); every last hop of the oracle tight (an edge whose
    use realises the distance) and equal to scipy's Dijkstra predecessor
    wherever the latter is the only tight one."""
    sp = pytest.importorskip("scipy.sparse.csgraph")
    n = 120
    W = graphgen.dense_graph_i64(n, seed=8, p=0.2, lo=1, hi=10 ** 12)
    D, P = oracle.fw_i64(W)
    Wf = np.where(W >= graphgen.INF_I64, np.inf, W.astype(np.float64))
    G = sp.csgraph_from_dense(Wf, null_value=np.inf)
    dist, pred = sp.shortest_path(G, method="D", directed=True, return_predecessors=True)
    reach = np.isfinite(dist)
    assert ((D < graphgen.INF_I64) == reach).all()
    np.testing.assert_array_equal(D[reach], dist[reach].astype(np.int64))
    off = reach & ~np.eye(n, dtype=bool)
    i, j = np.nonzero(off)
    u = P[i, j]
    assert (u >= 0).all()
    np.testing.assert_array_equal(D[i, u] + W[u, j], D[i, j])
    tight_scipy = D[i, pred[i, j]] + W[pred[i, j], j] == D[i, j]
    assert tight_scipy.all()
    # pairs where scipy's and the oracle's last hops differ have two tight last hops
    differ = P[i, j] != pred[i, j]
    assert differ.mean() < 0.01
    V = graphgen.dense_graph_f64(n, seed=9, p=0.3)
    Dv, Pv = oracle.fw_f64(V)
    G = sp.csgraph_from_dense(V, null_value=np.inf)
    dist, pred = sp.shortest_path(G, method="D", directed=True, return_predecessors=True)
    reach = np.isfinite(dist)
    assert (np.isfinite(Dv) == reach).all()
    np.testing.assert_allclose(Dv[reach], dist[reach], rtol=1e-13, atol=0)
    off = reach & ~np.eye(n, dtype=bool)
    i, j = np.nonzero(off)
    np.testing.assert_allclose(Dv[i, Pv[i, j]] + V[Pv[i, j], j], Dv[i, j], rtol=1e-13, atol=0)
    assert (Pv[i, j] == pred[i, j]).mean() > 0.99


def test_triangle_inequality():
    n = 64
    W = graphgen.dense_graph_i32(n, seed=9, p=0.2, lo=1, hi=30)
    D, _ = oracle.fw_i64(W)
    Dk = np.minimum(D, INF)
    via = (Dk[:, :, None] + Dk[None, :, :])  # via[i,k,j] = D_ik + D_kj
    assert (D[:, None, :] <= via).all()


def test_int_range_matches_float():
    """With small integer weights fp64 arithmetic is exact: both oracles agree."""
    n = 80
    W = graphgen.dense_graph_i32(n, seed=21, p=0.4, lo=1, hi=100)
    Wf = np.where(W >= INF, np.float32(np.inf), W.astype(np.float32))
    D, P = oracle.fw_i64(W)
    Df, Pf = oracle.fw_f64(Wf)
    reach = D < INF
    np.testing.assert_array_equal(Df[reach], D[reach].astype(np.float64))
    assert np.isinf(Df[~reach]).all()
    np.testing.assert_array_equal(Pf, P)


# ------------------------------------------------------------- certificate ---

def test_certificate_accepts_and_rejects():
    n = 50
    W = graphgen.dense_graph_i32(n, seed=31, p=0.3, lo=1, hi=20)
    D, P = oracle.fw_i64(W)
    D32 = D.astype(np.int32)
    assert oracle.certificate_i64(W, D32, P).sum() == 0
    rows = np.array([3, 17, 44])
    assert oracle.certificate_i64(W, D32[rows], P[rows], rows=rows).sum() == 0
    # planted faults, one per condition
    bad = D32.copy(); bad[2, 2] = 1
    assert oracle.certificate_i64(W, bad, P)[0] > 0
    i, j = np.argwhere((D > 0) & (D < INF) & (P != np.arange(n)[:, None]))[0]
    bad = D32.copy(); bad[i, j] += 1            # too long: some edge gives a shorter route
    c = oracle.certificate_i64(W, bad, P)
    assert c[1] + c[2] > 0
    bad = D32.copy(); bad[i, j] -= 1            # too short: not realised by its last hop
    assert oracle.certificate_i64(W, bad, P)[1] > 0
    badp = P.copy(); badp[i, j] = j             # self last hop
    assert oracle.certificate_i64(W, D32, badp)[1] > 0
    badp = P.copy(); badp[i, i] = (i + 1) % n   # pred on the diagonal
    assert oracle.certificate_i64(W, D32, badp)[3] > 0


def test_hops_and_margins():
    W, D, P = load_hand5()
    h = oracle.hops(P)
    expect = np.array([[0, 1, 2, 3, 2], [3, 0, 1, 2, 1], [2, 3, 0, 1, 2],
                       [1, 2, 3, 0, 1], [2, 3, 4, 1, 0]])
    np.testing.assert_array_equal(h, expect)
    m = oracle.lasthop_margin_i64(W, D, P)
    # 0 -> 2: last hop 1 (d 5); the alternative last hop is 0 itself (direct 7): gap 2
    assert m[0, 2] == 2
    # 0 -> 1 has no other in-neighbour than 0 except 3 (D03 + W31? no edge 3->1) -> no alternative
    assert m[0, 1] == np.iinfo(np.int64).max


def test_lasthop_margin_f64_hand_values():
    """The fp64 margin on the hand-worked graph read as fp32 weights (every
    weight and sum is exact in binary floating point), worked out by hand:
      0 -> 2: last hop 1 (d 5); the other in-neighbour of 2 is 0 (direct 7): 7 - 5 = 2
      0 -> 1: the only in-neighbour of 1 is 0, its last hop: no alternative (+inf)
      2 -> 4: last hop 3 (d 10 = 1 + 9); the other in-neighbour of 4 is 1 (d(2,1) 7 + 6 = 13): 3
      4 -> 0: last hop 3 (d 6); 0 has no other in-neighbour: +inf
      diagonal and unreachable entries: -1."""
    W, D, P = load_hand5()
    Wf = np.where(W >= INF, np.float32(np.inf), W.astype(np.float32)).astype(np.float32)
    Df, Pf = oracle.fw_f64(Wf)
    np.testing.assert_array_equal(Df, D.astype(np.float64))
    np.testing.assert_array_equal(Pf, P)
    m = oracle.lasthop_margin_f64(Wf, Df, Pf)
    assert m[0, 2] == 2.0
    assert np.isinf(m[0, 1]) and m[0, 1] > 0
    assert m[2, 4] == 3.0
    assert np.isinf(m[4, 0]) and m[4, 0] > 0
    assert (np.diag(m) == -1.0).all()
    # the integer margin agrees wherever both are finite
    mi = oracle.lasthop_margin_i64(W, D, P)
    fin = np.isfinite(m) & (mi != np.iinfo(np.int64).max)
    np.testing.assert_array_equal(m[fin], mi[fin].astype(np.float64))
    # a planted alternative: an edge 3 -> 2 of weight 6 gives 0 -> 2 a second
    # last hop at d(0,3) + 6 = 12, which does not lower the margin below 2
    W2 = Wf.copy(); W2[3, 2] = 6.0
    D2, P2 = oracle.fw_f64(W2)
    assert oracle.lasthop_margin_f64(W2, D2, P2)[0, 2] == 2.0
    # weight 0.5 on 3 -> 2 makes 0 -> 1 -> 2 -> 3 -> 2 irrelevant but 4 -> 3 -> 2
    # (2 + 0.5 = 2.5) beats 4 -> 3 -> 0 -> 1 -> 2 (11): last hop 3, margin to the
    # old last hop 1 (d(4,1) 8 + 3 = 11) is 8.5
    W3 = Wf.copy(); W3[3, 2] = 0.5
    D3, P3 = oracle.fw_f64(W3)
    assert D3[4, 2] == 2.5 and P3[4, 2] == 3
    assert oracle.lasthop_margin_f64(W3, D3, P3)[4, 2] == 8.5


# ---------------------------------------------------------------- gradient ---

def _unique_margin_instance(n, seed0, delta):
    for seed in range(seed0, seed0 + 400):
        W = graphgen.dense_graph_f32(n, seed=seed, p=0.3, kind=graphgen.KIND_ONE_TWO)
        # weights on a 2**-10 grid so W +- h (h = 2**-10) is exact in fp32
        W = np.where(np.isinf(W), W, np.round(W * 1024) / 1024).astype(np.float32)
        D, P = oracle.fw_f64(W)
        mg = oracle.lasthop_margin_f64(W, D, P)
        reach = np.isfinite(D) & ~np.eye(n, dtype=bool)
        if reach.sum() > n and (mg[reach] >= delta).all():
            return W, D, P
    pytest.skip("no instance with the required margin")


def test_grad_vs_finite_differences():
    n, h, delta = 16, 2.0 ** -10, 1e-2
    W, D, P = _unique_margin_instance(n, 100, delta)
    G = graphgen.adjoint_for(D, seed=7).astype(np.float64)
    GW = oracle.grad_f64(G, P)
    edges = np.argwhere(np.isfinite(W) & ~np.eye(n, dtype=bool))
    checked_nonzero = 0
    for (u, v) in edges:
        Wp = W.copy(); Wp[u, v] += h
        Wm = W.copy(); Wm[u, v] -= h
        Dp, _ = oracle.fw_f64(Wp)
        Dm, _ = oracle.fw_f64(Wm)
        fin = np.isfinite(D)
        fd = (G[fin] * (Dp[fin] - Dm[fin])).sum() / (2 * h)
        assert abs(fd - GW[u, v]) <= 1e-9 * (1 + abs(fd)), (u, v, fd, GW[u, v])
        checked_nonzero += GW[u, v] != 0
    assert checked_nonzero > 0
    # non-edges and the diagonal carry no gradient
    assert (GW[~np.isfinite(W)] == 0).all() and (np.diag(GW) == 0).all()


# ------------------------------------------- Fig. 1's P_ij <- k convention ---

def brute_force_mids(W, inf):
    """For every pair: the shortest distance and, over the shortest simple
    paths, the largest intermediate vertex of each (-1 for a single edge)."""
    n = W.shape[0]
    best = np.full((n, n), np.inf)
    mids_of = [[[] for _ in range(n)] for _ in range(n)]
    for s in range(n):
        best[s, s] = 0
        others = [v for v in range(n) if v != s]
        for L in range(1, n):
            for mids in itertools.permutations(others, L - 1):
                for t in others:
                    if t in mids:
                        continue
                    path = (s,) + mids + (t,)
                    ws = [W[a, b] for a, b in zip(path[:-1], path[1:])]
                    if any((np.isinf(w) if W.dtype.kind == "f" else w >= inf) for w in ws):
                        continue
                    c = float(sum(float(w) for w in ws))
                    top = max(mids) if mids else -1
                    if c < best[s, t]:
                        best[s, t] = c
                        mids_of[s][t] = [top]
                    elif c == best[s, t]:
                        mids_of[s][t].append(top)
    return best, mids_of


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("n", [5, 7])
def test_fw_k_brute_force(seed, n):
    """K[i][j] = the smallest over the shortest i -> j paths of the largest
    intermediate vertex; max_intermediate of the last-hop matrix is the largest
    intermediate vertex of one shortest path (the one P records)."""
    W = graphgen.dense_graph_i32(n, seed=seed, p=0.6, lo=1, hi=4)  # many ties
    best, mids_of = brute_force_mids(W, INF)
    Dk, K = oracle.fw_k_i64(W)
    D, P = oracle.fw_i64(W)
    np.testing.assert_array_equal(Dk, D)
    M = oracle.max_intermediate(P)
    ties = 0
    for s in range(n):
        for t in range(n):
            if s == t or np.isinf(best[s, t]):
                assert K[s, t] == -1 and M[s, t] == -1
                continue
            assert K[s, t] == min(mids_of[s][t]), (s, t, mids_of[s][t])
            assert M[s, t] in mids_of[s][t]
            if len(mids_of[s][t]) == 1:
                assert M[s, t] == K[s, t]
            ties += len(set(mids_of[s][t])) > 1
    assert ties > 0 or n == 5


@pytest.mark.parametrize("seed", [21, 22])
def test_fw_k_brute_force_float(seed):
    n = 7
    W = graphgen.dense_graph_f32(n, seed=seed, p=0.7)
    best, mids_of = brute_force_mids(W, None)
    Dk, K = oracle.fw_k_f64(W)
    D, P = oracle.fw_f64(W)
    np.testing.assert_array_equal(Dk, D)
    M = oracle.max_intermediate(P)
    for s in range(n):
        for t in range(n):
            if s == t or np.isinf(best[s, t]):
                assert K[s, t] == -1 and M[s, t] == -1
            elif len(mids_of[s][t]) == 1:
                assert K[s, t] == M[s, t] == mids_of[s][t][0]


def test_fw_k_closed_forms():
    """A path numbered upwards has its largest intermediate next to the
    target, one numbered downwards next to the source; a complete graph of
    unit weights has no intermediates at all."""
    n = 9
    Wu = np.full((n, n), INF, np.int32)
    np.fill_diagonal(Wu, 0)
    for k in range(n - 1):
        Wu[k, k + 1] = 2 + k % 3
    Wd = Wu.T.copy()                      # edges k + 1 -> k
    _, Ku = oracle.fw_k_i64(Wu)
    _, Kd = oracle.fw_k_i64(Wd)
    Mu = oracle.max_intermediate(oracle.fw_i64(Wu)[1])
    Md = oracle.max_intermediate(oracle.fw_i64(Wd)[1])
    for i in range(n):
        for j in range(n):
            up = j - 1 if j >= i + 2 else -1
            down = i - 1 if i >= j + 2 else -1
            assert Ku[i, j] == Mu[i, j] == up, (i, j)
            assert Kd[i, j] == Md[i, j] == down, (i, j)
    W1 = np.ones((12, 12), np.float32)
    np.fill_diagonal(W1, 0)
    assert (oracle.fw_k_f64(W1)[1] == -1).all()
    assert (oracle.max_intermediate(oracle.fw_f64(W1)[1]) == -1).all()


def test_fw_k_matches_max_intermediate_on_unique_paths():
    """Two independent routes to the same number on every pair with a unique
    shortest path: the k of Fig. 1's last improvement, and the walk of the
    last-hop path."""
    for n, seed in ((64, 3), (150, 4)):
        W = graphgen.dense_graph_i32(n, seed=seed, p=0.3, lo=1, hi=1000)
        Dk, K = oracle.fw_k_i64(W)
        D, P = oracle.fw_i64(W)
        M = oracle.max_intermediate(P)
        cnt = oracle.path_count_i64(W, D)
        uniq = (cnt == 1) & ~np.eye(n, dtype=bool) & (D < INF)
        assert uniq.sum() > n * n // 2
        np.testing.assert_array_equal(K[uniq], M[uniq])
        # elsewhere Fig. 1 keeps the smallest such vertex over the shortest paths
        assert (K <= M).all()


def test_max_intermediate_invalid_pred():
    """A last-hop matrix that does not lead back to the source yields -1."""
    P = np.array([[-1, 2, 1], [1, -1, 1], [2, 2, -1]], np.int32)  # 0: 1 <-> 2 cycle
    M = oracle.max_intermediate(P)
    assert M[0, 1] == -1 and M[0, 2] == -1
    assert M[1, 0] == -1 and M[1, 2] == -1 and M[2, 0] == -1 and M[2, 1] == -1
