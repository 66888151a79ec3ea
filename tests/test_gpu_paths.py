"""fw_paths: paths read back from a solved predecessor matrix on the GPU,
checked against the graph itself (every hop an edge, lengths summing to the
oracle's distance) and against a host walk of the same matrix."""
import numpy as np
import pytest

import graphgen
import oracle
from fwtest import INF, fw, gpu_solve

pytestmark = pytest.mark.gpu


def _host_walk(P, s, t, max_len):
    if s == t:
        return [s]
    if P[s, t] == -1:
        return None
    path = [t]
    v = t
    while v != s:
        v = int(P[s, v])
        path.append(v)
        if len(path) > len(P):
            raise AssertionError("pred is not a tree")
    return path[::-1]


def test_paths_match_graph_and_host_walk():
    import torch
    m = fw()
    n = 300
    W = graphgen.dense_graph_i32(n, seed=17, p=0.05, lo=1, hi=50)
    W[:250, 250:] = INF                                  # the last 50 vertices: out of reach of the rest
    Do, Po = oracle.fw_i64(W)
    D, P = gpu_solve(W, bs=64)
    np.testing.assert_array_equal(D.astype(np.int64), Do)
    rng = np.random.default_rng(5)
    src = rng.integers(0, n, 3000).astype(np.int32)
    dst = rng.integers(0, n, 3000).astype(np.int32)
    src[:10] = dst[:10]                                  # some trivial paths
    Pd = torch.from_numpy(P).cuda()
    out, lens = m.fw_paths(Pd, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    torch.cuda.synchronize()
    out, lens = out.cpu().numpy(), lens.cpu().numpy()
    unreachable = 0
    for q in range(len(src)):
        s, t = int(src[q]), int(dst[q])
        ref = _host_walk(P, s, t, n)
        if ref is None:
            assert lens[q] == 0 and Do[s, t] >= INF
            unreachable += 1
            continue
        assert lens[q] == len(ref), (q, s, t)
        path = out[q, :lens[q]].tolist()
        assert path == ref
        assert path[0] == s and path[-1] == t
        w = [int(W[a, b]) for a, b in zip(path[:-1], path[1:])]
        assert all(x < INF for x in w) and sum(w) == Do[s, t]
    assert unreachable > 0 and unreachable < len(src)


def test_paths_too_long_and_bad_ids():
    import torch
    m = fw()
    n = 64
    W = graphgen.dense_graph_i32(n, seed=3, p=0.0, lo=1, hi=5)   # no edges but a ring below
    for i in range(n):
        W[i, (i + 1) % n] = 1
    D, P = gpu_solve(W, bs=32)
    src = torch.tensor([0, 0, 5, -1, 0], dtype=torch.int32, device="cuda")
    dst = torch.tensor([63, 2, 5, 3, n], dtype=torch.int32, device="cuda")
    out, lens = m.fw_paths(torch.from_numpy(P).cuda(), src, dst, 3)
    assert lens.cpu().tolist() == [-1, 3, 1, -1, -1]         # 0 -> 63 has 64 vertices
    assert out[1].cpu().tolist() == [0, 1, 2] and out[2, 0].item() == 5
    out, lens = m.fw_paths(torch.from_numpy(P).cuda(), src[:1], dst[:1], n)
    assert lens.item() == n and out[0].cpu().tolist() == list(range(n))
