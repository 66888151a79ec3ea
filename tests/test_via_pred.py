"""The int32 solver's "via" predecessor encoding, checked on the CPU.

Remaining-tile (phase 4) tasks record "via k" (the intermediate vertex of the
improvement) instead of gathering the last hop of (k, j); pivot and panel
tasks copy such entries as they are, and one final pass follows each chain of
via codes down to a last hop.  This is exact because (k, j) cannot improve
again while (i, j) still records k: a strict improvement of (k, j) through a
later block improves (i, j) through that block too.

The test replays blocked FW (Sec. 2.3: phase 1 on the pivot tile, phases 2/3 on
its row and column, phase 4 on the rest; strict "<", first minimising k) twice
on small integer graphs -- once storing last hops throughout, once with the via
encoding and the final chain resolution -- and requires identical
predecessor matrices.  Plain Python loops, no GPU; independent of the oracle.
A second replay follows the persistent engine as it is now, whose panel tasks
record via codes too (a chain then takes at most two links per round).
"""
import numpy as np
import pytest

import graphgen

INF = graphgen.INF_I32


def _blocked_fw(W, bs, via):
    n = W.shape[0]
    D = W.astype(np.int64).copy()
    P = np.where((D < INF) & ~np.eye(n, dtype=bool), np.arange(n)[:, None], -1).astype(np.int64)

    def res(i, j):
        # follow the chain of via codes down to a last hop (each link points
        # to an improvement of an earlier round, so chains are short)
        p, hops = P[i, j], 0
        while p <= -2:
            p = P[-p - 2, j]
            hops += 1
            assert hops <= R, "via chain longer than the number of rounds"
        return p

    R = (n + bs - 1) // bs
    blk = lambda t: range(t * bs, min(n, (t + 1) * bs))
    for r in range(R):
        K = blk(r)
        # phase 1: in-place FW over block r (its own preds may be via codes:
        # they are copied as they are)
        for k in K:
            for i in K:
                for j in K:
                    s = D[i, k] + D[k, j]
                    if s < D[i, j]:
                        D[i, j], P[i, j] = s, P[k, j]
        piv_d = {(i, j): D[i, j] for i in K for j in K}
        piv_p = {(i, j): P[i, j] for i in K for j in K}
        # phases 2/3: row tiles (r, t) take their own preds, column tiles
        # (t, r) the pivot's (via codes copied as they are)
        for t in range(R):
            if t == r:
                continue
            for j in blk(t):
                old = {i: (D[i, j], P[i, j]) for i in K}
                for i in K:
                    best, bp = old[i]
                    for k in K:
                        s = piv_d[(i, k)] + old[k][0]
                        if s < best:
                            best, bp = s, old[k][1]
                    D[i, j], P[i, j] = best, bp
            for i in blk(t):
                old = {j: D[i, j] for j in K}
                for j in K:
                    best, bp, imp = old[j], P[i, j], False
                    for k in K:
                        s = old[k] + piv_d[(k, j)]
                        if s < best:
                            best, bp, imp = s, piv_p[(k, j)], True
                    if imp:
                        D[i, j], P[i, j] = best, bp
        # phase 4: first minimising k over the panels; via code or last hop
        for ti in range(R):
            for tj in range(R):
                if ti == r or tj == r:
                    continue
                for i in blk(ti):
                    for j in blk(tj):
                        best, bk = D[i, j], -1
                        for k in K:
                            s = D[i, k] + D[k, j]
                            if s < best:
                                best, bk = s, k
                        if bk >= 0:
                            D[i, j] = best
                            P[i, j] = -(bk + 2) if via else P[bk, j]
    if via:
        P = np.array([[res(i, j) for j in range(n)] for i in range(n)])
    return D, P


@pytest.mark.parametrize("n,bs,p,hi,seed", [(23, 4, 0.5, 20, 1), (30, 8, 0.3, 9, 2),
                                            (28, 5, 0.8, 3, 3), (17, 3, 0.25, 50, 4),
                                            (40, 4, 0.6, 2, 5), (33, 2, 0.15, 100, 6)])
def test_via_encoding_matches_last_hops(n, bs, p, hi, seed):
    W = graphgen.dense_graph_i32(n, seed=seed, p=p, lo=1, hi=hi)
    D0, P0 = _blocked_fw(W, bs, via=False)
    D1, P1 = _blocked_fw(W, bs, via=True)
    np.testing.assert_array_equal(D0, D1)
    np.testing.assert_array_equal(P0, P1)
    # and the replay is a shortest-path solver at all (distances of plain FW)
    Dref = W.astype(np.int64).copy()
    for k in range(n):
        Dref = np.minimum(Dref, Dref[:, k:k + 1] + Dref[k:k + 1, :])
    np.testing.assert_array_equal(D0, Dref)



def _engine_replay(W, bs, via):
    """The persistent engine's schedule as it is now: panels as products with
    the closed pivot that record via codes like the remaining tiles (or
    gather last hops, via=False)."""
    n = W.shape[0]
    D = W.astype(np.int64).copy()
    P = np.where((D < INF) & ~np.eye(n, dtype=bool), np.arange(n)[:, None], -1).astype(np.int64)
    R = (n + bs - 1) // bs
    blk = lambda t: list(range(t * bs, min(n, (t + 1) * bs)))

    def res(i, j):
        p, hops = P[i, j], 0
        while p <= -2:
            p = P[-p - 2, j]
            hops += 1
            assert hops <= 2 * R + 2, "via chain longer than two links per round"
        return p

    for r in range(R):
        K = blk(r)
        for k in K:
            for i in K:
                for j in K:
                    s = D[i, k] + D[k, j]
                    if s < D[i, j]:
                        D[i, j], P[i, j] = s, P[k, j]
        piv_d = {(i, j): D[i, j] for i in K for j in K}
        piv_p = {(i, j): P[i, j] for i in K for j in K}
        for t in range(R):
            if t == r:
                continue
            for j in blk(t):                       # row tile (r, t)
                old = {i: (D[i, j], P[i, j]) for i in K}
                for i in K:
                    best, bk = old[i][0], -1
                    for k in K:
                        s = piv_d[(i, k)] + old[k][0]
                        if s < best:
                            best, bk = s, k
                    if bk >= 0:
                        D[i, j] = best
                        P[i, j] = -(bk + 2) if via else old[bk][1]
            for i in blk(t):                       # column tile (t, r)
                old = {j: D[i, j] for j in K}
                for j in K:
                    best, bk = old[j], -1
                    for k in K:
                        s = old[k] + piv_d[(k, j)]
                        if s < best:
                            best, bk = s, k
                    if bk >= 0:
                        D[i, j] = best
                        P[i, j] = -(bk + 2) if via else piv_p[(bk, j)]
        for ti in range(R):
            for tj in range(R):
                if ti == r or tj == r:
                    continue
                for i in blk(ti):
                    for j in blk(tj):
                        best, bk = D[i, j], -1
                        for k in K:
                            s = D[i, k] + D[k, j]
                            if s < best:
                                best, bk = s, k
                        if bk >= 0:
                            D[i, j] = best
                            P[i, j] = -(bk + 2) if via else P[bk, j]
    if via:
        P = np.array([[res(i, j) for j in range(n)] for i in range(n)])
    return D, P


@pytest.mark.parametrize("n,bs,p,lo,hi,seed", [(23, 4, 0.5, 1, 20, 1), (30, 8, 0.3, 0, 9, 2),
                                               (28, 5, 0.8, 0, 3, 3), (17, 3, 0.25, 1, 50, 4),
                                               (40, 4, 0.6, 0, 2, 5), (33, 8, 0.15, 1, 100, 6)])
def test_engine_via_codes(n, bs, p, lo, hi, seed):
    """Panel via codes resolve to the last hops that gathering gives, chains
    stay within two links per round (zero weights included), and every
    resolved last hop is tight."""
    W = graphgen.dense_graph_i32(n, seed=seed, p=p, lo=lo, hi=hi)
    D0, P0 = _engine_replay(W, bs, via=False)
    D1, P1 = _engine_replay(W, bs, via=True)
    np.testing.assert_array_equal(D0, D1)
    np.testing.assert_array_equal(P0, P1)
    Dref = W.astype(np.int64).copy()
    for k in range(n):
        Dref = np.minimum(Dref, Dref[:, k:k + 1] + Dref[k:k + 1, :])
    np.testing.assert_array_equal(D0, Dref)
    for i in range(n):
        for j in range(n):
            if i == j or D0[i, j] >= INF:
                assert P1[i, j] == -1 or i == j
                continue
            u = P1[i, j]
            assert 0 <= u < n and u != j and D0[i, u] + W[u, j] == D0[i, j], (i, j, u)
