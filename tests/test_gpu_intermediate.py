"""fw_intermediate: the paper's Fig. 1 path bookkeeping (P_ij = k) from a
last-hop matrix, on the GPU.

* bit-exact against the oracle's walk of the same (oracle-made) last-hop
  matrix, at sizes spanning several warps per row and ragged tails, with
  padded rows, batches and in place;
* end to end: a GPU solve, then fw_intermediate, equal to Fig. 1's k (the
  oracle's own FW loop) on every pair with a unique shortest path, and a
  valid split point (D_ik + D_kj = D_ij) everywhere else;
* the largest supported n (57344) on a closed form.
"""
import numpy as np
import pytest

import graphgen
import oracle
from fwtest import INF, fw, gpu_solve

pytestmark = pytest.mark.gpu


def _dev(a, ld=None):
    import torch
    n = a.shape[-1]
    ld = ld or n
    buf = torch.full(a.shape[:-1] + (ld,), -77, dtype=torch.int32, device="cuda")
    v = buf[..., :n]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return buf, v


@pytest.mark.parametrize("n,p,seed,pad", [(1, 0.5, 1, 0), (2, 1.0, 2, 3), (37, 0.2, 3, 3),
                                          (300, 0.05, 4, 4), (1000, 0.01, 5, 0),
                                          (1000, 0.5, 6, 8)])
def test_matches_oracle_walk(n, p, seed, pad):
    import torch
    m = fw()
    W = graphgen.dense_graph_i32(n, seed=seed, p=p, lo=1, hi=100)
    if n > 20:
        W[: n // 2, n - n // 5:] = INF            # some pairs out of reach
    _, Po = oracle.fw_i64(W)
    Mo = oracle.max_intermediate(Po)
    buf, P = _dev(Po, n + pad)
    M = m.fw_intermediate(P)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(M.cpu().numpy(), Mo)
    assert (buf[:, n:] == -77).all()               # padding of pred untouched
    # in place: out = pred
    m.fw_intermediate(P, out=P)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(P.cpu().numpy(), Mo)
    assert (buf[:, n:] == -77).all()


def test_batched_strided():
    import torch
    m = fw()
    n, B = 257, 3
    Ps, Ms = [], []
    for b in range(B):
        W = graphgen.dense_graph_i32(n, seed=40 + b, p=0.03 * (b + 1), lo=1, hi=30)
        Ps.append(oracle.fw_i64(W)[1])
        Ms.append(oracle.max_intermediate(Ps[-1]))
    buf, P = _dev(np.stack(Ps), n + 3)
    M = m.fw_intermediate(P)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(M.cpu().numpy(), np.stack(Ms))


def test_invalid_pred_rows():
    """Entries outside [0, n), self-loops and a cycle that never reaches the
    source: the same -1s as the oracle's bounded walk."""
    import torch
    m = fw()
    n = 70
    rng = np.random.default_rng(9)
    P = rng.integers(-3, n + 3, (n, n)).astype(np.int32)
    np.fill_diagonal(P, -1)
    Mo = oracle.max_intermediate(P)
    _, Pd = _dev(P)
    M = m.fw_intermediate(Pd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(M.cpu().numpy(), Mo)


@pytest.mark.parametrize("n,p,bs", [(700, 0.05, 64), (1500, 0.3, 128)])
def test_end_to_end_is_fig1_k_on_unique_paths(n, p, bs):
    import torch
    m = fw()
    W = graphgen.dense_graph_i32(n, seed=n, p=p, lo=1, hi=60)
    Dk, K = oracle.fw_k_i64(W)
    D, P = gpu_solve(W, bs=bs)
    np.testing.assert_array_equal(D.astype(np.int64), Dk)
    M = m.fw_intermediate(torch.from_numpy(P).cuda()).cpu().numpy()
    cnt = oracle.path_count_i64(W, Dk)
    off = ~np.eye(n, dtype=bool)
    reach = (Dk < INF) & off
    uniq = reach & (cnt == 1)
    assert uniq.sum() > 0.3 * reach.sum()
    np.testing.assert_array_equal(M[uniq], K[uniq])
    # elsewhere: -1 only where the recorded path is one edge, else a vertex
    # on a shortest path, no smaller than Fig. 1's (the smallest such)
    edge = reach & (P == np.arange(n)[:, None])
    assert (M[edge] == -1).all()
    rest = reach & ~edge
    i, j = np.nonzero(rest)
    k = M[rest]
    assert (k >= 0).all() and (k != i).all() and (k != j).all()
    np.testing.assert_array_equal(Dk[i, k] + Dk[k, j], Dk[i, j])
    assert (k >= K[rest]).all()
    assert (M[~reach] == -1).all()


def test_end_to_end_fp32():
    """fp32 weights on a 1/16 grid: every path sum is exact in fp32, so the
    fp32 solve sees the same ties as the integer graph it scales."""
    import torch
    m = fw()
    n = 900
    Wi = graphgen.dense_graph_i32(n, seed=31, p=0.1, lo=16, hi=512)
    Wf = np.where(Wi >= INF, np.inf, Wi / 16.0).astype(np.float32)
    Dk, K = oracle.fw_k_f64(Wf)
    D, P = gpu_solve(Wf)
    np.testing.assert_array_equal(D.astype(np.float64), Dk)
    M = m.fw_intermediate(torch.from_numpy(P).cuda()).cpu().numpy()
    Di, _ = oracle.fw_i64(Wi)
    cnt = oracle.path_count_i64(Wi, Di)
    uniq = np.isfinite(Dk) & ~np.eye(n, dtype=bool) & (cnt == 1)
    assert uniq.sum() > 0.3 * np.isfinite(Dk).sum()
    np.testing.assert_array_equal(M[uniq], K[uniq])


def test_largest_n_closed_form():
    """n = 57344 (every row 224 KB of shared memory): pred with the last hop
    of an odd vertex v its even neighbour v - 1, of an even vertex the source,
    so the largest intermediate of an odd v is v - 1 (unless that is the
    source) and every other pair has none."""
    import torch
    m = fw()
    n = 57344
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    i = torch.arange(n, dtype=torch.int32, device="cuda")[:, None]
    odd = (v % 2 == 1)[None, :]
    P = torch.where(odd, (v - 1)[None, :], i)
    P.fill_diagonal_(-1)
    M = m.fw_intermediate(P)
    exp = torch.where(odd & ((v - 1)[None, :] != i), (v - 1)[None, :], torch.full_like(P, -1))
    exp.fill_diagonal_(-1)
    assert torch.equal(M, exp)
    del P, M, exp
    torch.cuda.empty_cache()
