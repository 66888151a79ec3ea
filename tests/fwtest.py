"""Helpers shared by the GPU parity tests (not collected as tests)."""
from __future__ import annotations

import functools

import numpy as np

import graphgen
import oracle

INF = graphgen.INF_I32
CANARY_I = np.int32(-123456789)
CANARY_F = np.float32(-7.25)


def _torch_dtype_and_canary(dtype):
    """(torch dtype, padding canary) of a numpy weight dtype."""
    import torch
    table = {np.dtype(np.int32): (torch.int32, int(CANARY_I)),
             np.dtype(np.float32): (torch.float32, float(CANARY_F)),
             np.dtype(np.int64): (torch.int64, -123456789123),
             np.dtype(np.float64): (torch.float64, -7.25)}
    return table[np.dtype(dtype)]


def fw():
    import paper_2403_18619_gb300 as m
    return m


def gpu_solve(W: np.ndarray, *, bs=0, driver=0, packed=1, extra_ld=0, lookahead=-1, grid=0,
              stream=None, check_canary=True, tile_tma=1):
    """Solve a host matrix on the GPU through the C ABI; returns host (D, P)."""
    import torch
    m = fw()
    n = W.shape[0]
    ld = m.padded(n) + extra_ld
    tdt, canary = _torch_dtype_and_canary(W.dtype)
    Dbuf = torch.full((n, ld), canary, dtype=tdt, device="cuda")
    Pbuf = torch.full((n, ld), -987654, dtype=torch.int32, device="cuda")
    D, P = Dbuf[:, :n], Pbuf[:, :n]
    D.copy_(torch.from_numpy(np.ascontiguousarray(W)))
    opt = m.Options.default(bs=bs, driver=driver, packed_keys=packed, lookahead=lookahead,
                            grid=grid, tile_tma=tile_tma)
    m.fw_solve_ex(D, P, opt, stream)
    m.fw_sync_status(stream)
    Dh, Ph = Dbuf.cpu().numpy(), Pbuf.cpu().numpy()
    if check_canary and ld > n:
        assert (Dh[:, n:] == canary).all(), "dist padding was written"
        assert (Ph[:, n:] == -987654).all(), "pred padding was written"
    return Dh[:, :n].copy(), Ph[:, :n].copy()


@functools.lru_cache(maxsize=32)
def _oracle_int(key):
    n, seed, p, lo, hi = key
    W = graphgen.dense_graph_i32(n, seed=seed, p=p, lo=lo, hi=hi)
    D, P = oracle.fw_i64(W)
    cnt = oracle.path_count_i64(W, D)
    return W, D, P, cnt


def int_case(n, seed, p, lo, hi):
    return _oracle_int((n, seed, p, lo, hi))


def check_int_full(W, D, P, Do, Po, cnt):
    """Bit-exact distances, predecessors on unique paths, certificate elsewhere."""
    n = W.shape[0]
    assert D.dtype == np.int32
    mism = np.argwhere(D.astype(np.int64) != Do)
    assert len(mism) == 0, "dist differs at %d entries, first %s: gpu %d oracle %d" % (
        len(mism), mism[0].tolist(), D[tuple(mism[0])], Do[tuple(mism[0])])
    uniq = (cnt == 1) & ~np.eye(n, dtype=bool)
    bad = np.argwhere((P != Po) & uniq)
    assert len(bad) == 0, "pred differs on %d unique-path pairs, first %s: gpu %d oracle %d" % (
        len(bad), bad[0].tolist(), P[tuple(bad[0])], Po[tuple(bad[0])])
    cert = oracle.certificate_i64(W, D, P)
    assert cert.sum() == 0, "certificate violations %s" % cert.tolist()


def check_int_rows(W, D, P, rows):
    """Sampled rows against Dijkstra from each sampled source."""
    Dd, Pd = oracle.dijkstra_i64(W, rows)
    np.testing.assert_array_equal(D[rows].astype(np.int64), Dd)
    cnt = oracle.path_count_i64(W, Dd, rows=rows)
    uniq = cnt == 1
    uniq[np.arange(len(rows)), rows] = False
    assert (P[rows][uniq] == Pd[uniq]).all()
    cert = oracle.certificate_i64(W, D[rows], P[rows], rows=rows)
    assert cert.sum() == 0, cert.tolist()
    return int(uniq.sum())


def check_f32(W, D, P, Do, Po, rows=None):
    """fp32 distances within 1e-6 * hops relative of the fp64 oracle; predecessors
    equal where the oracle's last hop wins by more than twice that tolerance."""
    rows_idx = np.arange(W.shape[0]) if rows is None else np.asarray(rows)
    Dg, Pg = D[rows_idx], P[rows_idx]
    reach = np.isfinite(Do)
    assert (np.isfinite(Dg) == reach).all(), "reachability differs"
    hops = oracle.hops(Po, rows=None if rows is None else rows_idx)
    tol = 1e-6 * np.maximum(hops, 1) * np.abs(Do)
    err = np.abs(Dg.astype(np.float64) - Do)
    err[~reach] = 0
    worst = np.unravel_index(np.argmax(err - tol), err.shape)
    assert (err <= tol).all(), "fp32 error %g > tol %g at %s" % (err[worst], tol[worst], worst)
    mg = oracle.lasthop_margin_f64(W, Do, Po, rows=None if rows is None else rows_idx)
    safe = reach & (mg > 2 * tol) & (hops > 0)
    assert (Pg[safe] == Po[safe]).all(), "fp32 pred differs on margin-safe pairs"
    return int(safe.sum())


def check_f32_dist(W, D, Do, Po):
    """fp32 distances only (a distance-only solve): within 1e-6 * hops relative
    of the fp64 oracle, reachability exact."""
    reach = np.isfinite(Do)
    assert (np.isfinite(D) == reach).all(), "reachability differs"
    hops = oracle.hops(Po)
    tol = 1e-6 * np.maximum(hops, 1) * np.abs(Do)
    err = np.abs(D.astype(np.float64) - Do)
    err[~reach] = 0
    worst = np.unravel_index(np.argmax(err - tol), err.shape)
    assert (err <= tol).all(), "fp32 error %g > tol %g at %s" % (err[worst], tol[worst], worst)


def gpu_solve_dist_only(W: np.ndarray, *, bs=0, driver=0, packed=1, extra_ld=0):
    """Distance-only solve (pred = NULL) through the C ABI; returns host D and
    checks that the padding columns were left alone."""
    import torch
    m = fw()
    n = W.shape[0]
    ld = m.padded(n) + extra_ld
    tdt, canary = _torch_dtype_and_canary(W.dtype)
    Dbuf = torch.full((n, ld), canary, dtype=tdt, device="cuda")
    D = Dbuf[:, :n]
    D.copy_(torch.from_numpy(np.ascontiguousarray(W)))
    m.fw_solve_ex(D, None, m.Options.default(bs=bs, driver=driver, packed_keys=packed))
    m.fw_sync_status()
    Dh = Dbuf.cpu().numpy()
    if ld > n:
        assert (Dh[:, n:] == canary).all(), "dist padding was written"
    return Dh[:, :n].copy()


def check_pred_tight_int(W, Do, Pg, Po, inf=INF):
    """Predecessors against the full int64 oracle: equal to the oracle's last
    hop, or else another last hop u that is tight (an edge u -> j with
    D[i][u] + W[u][j] == D[i][j]).  A second tight last hop means a second
    shortest path, so on every pair with a unique shortest path the two agree,
    and elsewhere the GPU's last hop realises the distance.  Returns the number
    of pairs where they differ."""
    n = W.shape[0]
    i, j = np.nonzero(Pg != Po)
    if len(i) == 0:
        return 0
    u = Pg[i, j].astype(np.int64)
    assert ((u >= 0) & (u < n) & (u != j)).all(), "pred out of range where it differs"
    w = W[u, j].astype(np.int64)
    assert (w < inf).all(), "pred is not an in-neighbour where it differs"
    bad = Do[i, u] + w != Do[i, j]
    assert not bad.any(), "pred not tight at %d pairs, first (%d, %d)" % (
        bad.sum(), i[bad][0], j[bad][0])
    return len(i)


def check_pred_near_tight_f32(W, Do, Pg, Po, tol):
    """fp32 predecessors against the full fp64 oracle: equal to the oracle's
    last hop, or else another last hop u whose path is within 2 * tol of the
    shortest distance in fp64 (D[i][u] + W[u][j] <= D[i][j] + 2 tol[i][j]).
    The oracle's margin of such a pair is then at most 2 tol, so on every
    margin-safe pair the two agree.  Returns the number of differing pairs."""
    n = W.shape[0]
    i, j = np.nonzero(Pg != Po)
    if len(i) == 0:
        return 0
    u = Pg[i, j].astype(np.int64)
    assert ((u >= 0) & (u < n) & (u != j)).all(), "pred out of range where it differs"
    w = W[u, j].astype(np.float64)
    assert np.isfinite(w).all(), "pred is not an in-neighbour where it differs"
    gap = Do[i, u] + w - Do[i, j]
    bad = gap > 2 * tol[i, j]
    assert not bad.any(), "pred not near-tight at %d pairs, first (%d, %d) gap %g tol %g" % (
        bad.sum(), i[bad][0], j[bad][0], gap[bad][0], tol[i[bad][0], j[bad][0]])
    return len(i)
