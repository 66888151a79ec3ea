"""The single-graph multi-GPU schedule through the CUDA tile calls
(fw_tile_closure, fw_tile_minplus, fw_block_init_pred), every rank of the
grid emulated in this process on one GPU, in lockstep (a broadcast is a device
copy; no kernel waits for another rank's), against the full oracle; and the
tile calls alone against the test-side CPU tile operations."""
import numpy as np
import pytest

import graphgen
import oracle
from fwtest import check_pred_near_tight_f32, check_pred_tight_int, fw

pytestmark = pytest.mark.gpu


def _run(W, pr, pc, bs, with_pred=True):
    import torch
    from paper_2403_18619_gb300 import distributed as fd
    grid = fd.Grid(W.shape[0], bs, pr, pc)
    states = []
    for r in range(grid.world):
        D = torch.from_numpy(fd.scatter_block(W, grid, r)).cuda()
        P = torch.empty(D.shape, dtype=torch.int32, device="cuda") if with_pred else None
        states.append(fd.RankState.create(r, grid, D, P))
    fd.solve_block_cyclic(states, grid, fd.LocalComm(grid), fd.CudaTileOps)
    fw().fw_sync_status()
    D = fd.gather_blocks([s.D.cpu().numpy() for s in states], grid, fill=0)
    P = fd.gather_blocks([s.P.cpu().numpy() for s in states], grid) if with_pred else None
    return D, P


@pytest.mark.parametrize("pr,pc,bs", [(1, 1, 64), (2, 2, 32), (1, 3, 64), (2, 1, 128), (3, 3, 32)])
def test_int32_grids(pr, pc, bs):
    n = 700  # ragged for every block size here
    W = graphgen.dense_graph_i32(n, seed=pr * 10 + pc, p=0.3, lo=1, hi=200)
    Do, Po = oracle.fw_i64(W)
    D, P = _run(W, pr, pc, bs)
    np.testing.assert_array_equal(D.astype(np.int64), Do)
    check_pred_tight_int(W, Do, P, Po)


@pytest.mark.parametrize("kind,bs", [("f32", 64), ("f64", 32), ("i64", 64)])
def test_other_dtypes(kind, bs):
    n = 500
    if kind == "f32":
        W = graphgen.dense_graph_f32(n, seed=3, p=0.4)
    elif kind == "f64":
        W = graphgen.dense_graph_f64(n, seed=3, p=0.4)
    else:
        W = graphgen.dense_graph_i64(n, seed=3, p=0.4, lo=1, hi=10 ** 12)
    D, P = _run(W, 2, 2, bs)
    if kind == "i64":
        Do, Po = oracle.fw_i64(W)
        np.testing.assert_array_equal(D, Do)
        check_pred_tight_int(W, Do, P, Po, inf=graphgen.INF_I64)
        return
    Do, Po = oracle.fw_f64(W)
    reach = np.isfinite(Do)
    assert (np.isfinite(D) == reach).all()
    tol = (1e-6 if kind == "f32" else 1e-15) * np.maximum(oracle.hops(Po), 1) * np.abs(Do)
    tol[~reach] = 0
    err = np.abs(D.astype(np.float64) - Do)
    err[~reach] = 0
    assert (err <= tol).all()
    check_pred_near_tight_f32(W, Do, P, Po, tol)


def test_distance_only_and_negative_cycle():
    import torch
    m = fw()
    W = graphgen.dense_graph_i32(300, seed=5, p=0.3, lo=1, hi=20)
    Do, _ = oracle.fw_i64(W)
    D, _ = _run(W, 2, 2, 32, with_pred=False)
    np.testing.assert_array_equal(D.astype(np.int64), Do)
    Wn = W.copy()
    Wn[40, 41], Wn[41, 42], Wn[42, 40] = 1, 1, -10
    with pytest.raises(m.FWError) as e:
        _run(Wn, 2, 2, 32)
    assert e.value.code == 4
    m.fw_sync_status()


@pytest.mark.parametrize("dtype", ["i32", "f32", "f64"])
def test_tile_calls_match_cpu_tile_ops(dtype):
    """fw_tile_closure and fw_tile_minplus on one input, in the three aliasing
    forms the schedule uses, against the CPU tile operations (exact for the
    integer and the integer-valued inputs here)."""
    import torch
    from tileops_cpu import NumpyTileOps
    m = fw()
    bs, tm, tn = 32, 3, 4
    rng = np.random.default_rng(7)
    np_t = {"i32": np.int32, "f32": np.float32, "f64": np.float64}[dtype]

    def rand(shape):
        return rng.integers(1, 60, size=shape).astype(np_t)

    piv = rand((bs, bs)); np.fill_diagonal(piv, 0)
    pivP = rng.integers(0, 1000, size=(bs, bs)).astype(np.int32)
    C = rand((tm * bs, tn * bs)); Pc = rng.integers(0, 1000, size=C.shape).astype(np.int32)
    A = rand((tm * bs, bs))
    B = rand((bs, tn * bs)); Pb = rng.integers(0, 1000, size=B.shape).astype(np.int32)
    cases = {
        "closure": None,
        "remaining": (C, Pc, A, B, Pb, 1, 2),
        "row_panel": (C[:bs], Pc[:bs], piv, None, None, -1, 1),
        "col_panel": (C[:, :bs], Pc[:, :bs], None, piv, pivP, 2, -1),
    }
    for name, args in cases.items():
        if name == "closure":
            ref_d, ref_p = torch.from_numpy(piv.copy()), torch.from_numpy(pivP.copy())
            NumpyTileOps.closure(ref_d, ref_p, bs)
            d, p = torch.from_numpy(piv.copy()).cuda(), torch.from_numpy(pivP.copy()).cuda()
            m.fw_tile_closure(d, p, bs)
            m.fw_sync_status()
            np.testing.assert_array_equal(d.cpu().numpy(), ref_d.numpy())
            np.testing.assert_array_equal(p.cpu().numpy(), ref_p.numpy())
            continue
        c0, p0, a0, b0, pb0, si, sj = args
        c_ref = torch.from_numpy(np.ascontiguousarray(c0).copy())
        p_ref = torch.from_numpy(np.ascontiguousarray(p0).copy())
        c_dev, p_dev = c_ref.clone().cuda(), p_ref.clone().cuda()
        if name == "row_panel":      # B = C, Pb = Pc
            NumpyTileOps.minplus(c_ref, p_ref, torch.from_numpy(a0), c_ref, p_ref, bs, si, sj)
            m.fw_tile_minplus(c_dev, p_dev, torch.from_numpy(a0).cuda(), c_dev, p_dev, bs, si, sj)
        elif name == "col_panel":    # A = C
            bb, pp = torch.from_numpy(b0), torch.from_numpy(pb0)
            NumpyTileOps.minplus(c_ref, p_ref, c_ref, bb, pp, bs, si, sj)
            m.fw_tile_minplus(c_dev, p_dev, c_dev, bb.cuda(), pp.cuda(), bs, si, sj)
        else:
            aa, bb, pp = (torch.from_numpy(x) for x in (a0, b0, pb0))
            NumpyTileOps.minplus(c_ref, p_ref, aa, bb, pp, bs, si, sj)
            m.fw_tile_minplus(c_dev, p_dev, aa.cuda(), bb.cuda(), pp.cuda(), bs, si, sj)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(c_dev.cpu().numpy(), c_ref.numpy(), err_msg=name)
        np.testing.assert_array_equal(p_dev.cpu().numpy(), p_ref.numpy(), err_msg=name)
