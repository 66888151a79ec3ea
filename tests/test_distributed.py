"""The single-graph multi-GPU schedule (2-D block-cyclic tiles, a pivot and
two panel broadcasts per round) on the CPU: gloo ranks (world size 2 and 4)
and the in-process lockstep emulation, with test-side CPU tile operations,
against the full oracle.  Checks the owner map, the local blocks, the order
of the phases and the broadcasts' roots and groups."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

import graphgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graph(kind, n):
    if kind == "i32":
        return graphgen.dense_graph_i32(n, seed=17, p=0.3, lo=1, hi=50)
    if kind == "f32":
        return graphgen.dense_graph_f32(n, seed=18, p=0.3)
    return graphgen.dense_graph_f64(n, seed=19, p=0.3)


def _check(W, D, P, with_pred=True):
    n = W.shape[0]
    if W.dtype.kind == "i":
        Do, Po = oracle.fw_i64(W)
        np.testing.assert_array_equal(D.astype(np.int64), Do)
        if with_pred:
            from fwtest import check_pred_tight_int
            check_pred_tight_int(W, Do, P, Po)
    else:
        Do, Po = oracle.fw_f64(W)
        reach = np.isfinite(Do)
        assert (np.isfinite(D) == reach).all()
        hops = oracle.hops(Po)
        rel = 1e-6 if W.dtype == np.float32 else 1e-15
        tol = rel * np.maximum(hops, 1) * np.abs(Do)
        tol[~reach] = 0
        err = np.abs(D.astype(np.float64) - Do)
        err[~reach] = 0
        assert (err <= tol).all()
        if with_pred:
            from fwtest import check_pred_near_tight_f32
            check_pred_near_tight_f32(W, Do, P, Po, tol)


def _rank_main(rank, world, port, pr, pc, kind, n, bs, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    from paper_2403_18619_gb300 import distributed as fd
    from tileops_cpu import NumpyTileOps
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = fd.Grid(n, bs, pr, pc)
        W = _graph(kind, n)
        D = torch.from_numpy(fd.scatter_block(W, grid, rank))
        P = torch.empty(D.shape, dtype=torch.int32)
        st = fd.RankState.create(rank, grid, D, P)
        fd.solve_block_cyclic([st], grid, fd.TorchComm(grid), NumpyTileOps)
        dist.barrier()
        q.put((rank, D.numpy().copy(), P.numpy().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("pr,pc,kind,n,bs", [
    (1, 2, "i32", 200, 32),      # ragged: 200 = 6 * 32 + 8
    (2, 1, "f32", 150, 32),
    (2, 2, "i32", 230, 32),
    (2, 2, "f64", 100, 16 * 2),
])
def test_gloo_ranks_match_the_oracle(pr, pc, kind, n, bs):
    world = pr * pc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, pr, pc, kind, n, bs, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(world):
        rank, D, P = q.get(timeout=300)
        got[rank] = (D, P)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    from paper_2403_18619_gb300 import distributed as fd
    grid = fd.Grid(n, bs, pr, pc)
    D = fd.gather_blocks([got[r][0] for r in range(world)], grid, fill=0)
    P = fd.gather_blocks([got[r][1] for r in range(world)], grid)
    _check(_graph(kind, n), D, P)


@pytest.mark.parametrize("pr,pc", [(1, 1), (2, 3), (3, 2), (4, 4)])
@pytest.mark.parametrize("with_pred", [True, False])
def test_lockstep_emulation_matches_the_oracle(pr, pc, with_pred):
    """Every rank in this process (LocalComm): the same schedule; 4 x 4 on an
    R = 5 grid leaves ranks with fewer tile rows than others."""
    import torch
    from paper_2403_18619_gb300 import distributed as fd
    from tileops_cpu import NumpyTileOps
    n, bs = 150, 32
    W = _graph("i32", n)
    grid = fd.Grid(n, bs, pr, pc)
    states = []
    for r in range(grid.world):
        D = torch.from_numpy(fd.scatter_block(W, grid, r))
        P = torch.empty(D.shape, dtype=torch.int32) if with_pred else None
        states.append(fd.RankState.create(r, grid, D, P))
    fd.solve_block_cyclic(states, grid, fd.LocalComm(grid), NumpyTileOps)
    D = fd.gather_blocks([s.D.numpy() for s in states], grid, fill=0)
    P = fd.gather_blocks([s.P.numpy() for s in states], grid) if with_pred else None
    _check(W, D, P, with_pred)


def test_grid_owner_map_and_blocks():
    from paper_2403_18619_gb300 import distributed as fd
    g = fd.Grid(n=230, bs=32, pr=2, pc=3)
    assert g.R == 8 and g.world == 6
    # every tile has exactly one owner, and it is in the owner's local lists
    seen = {}
    for I in range(g.R):
        for J in range(g.R):
            o = g.owner(I, J)
            prow, pcol = g.coords(o)
            assert I in g.tile_rows(prow) and J in g.tile_cols(pcol)
            seen[(I, J)] = o
    assert len(seen) == g.R * g.R
    assert sum(len(g.tile_rows(a)) for a in range(g.pr)) == g.R
    assert sum(len(g.tile_cols(c)) for c in range(g.pc)) == g.R
    W = graphgen.dense_graph_i32(230, seed=1, p=0.5, lo=1, hi=9)
    blocks = [fd.scatter_block(W, g, r) for r in range(g.world)]
    np.testing.assert_array_equal(fd.gather_blocks(blocks, g), W)
    # padding vertices are isolated with a zero diagonal
    b = blocks[g.owner(7, 7)]
    lr, lc = 7 // g.pr, 7 // g.pc
    tile = b[lr * 32:(lr + 1) * 32, lc * 32:(lc + 1) * 32]
    real = 230 - 7 * 32
    assert (np.diag(tile)[real:] == 0).all()
    assert (tile[real:, :][~np.eye(32, dtype=bool)[real:, :]] == graphgen.INF_I32).all()
