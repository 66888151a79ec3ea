"""The 64-bit element types (the paper's double-precision runs, Sec. 4, and
int64 weights) against the full oracle (plain FW of Sec. 2.3, Fig. 1, in
int64 / fp64): every distance (int64 bit-exact; fp64 within 1e-15 * hops
relative, hops of the oracle's paths) and every predecessor (the oracle's, or
another tight / near-tight last hop, which makes the pair non-unique / not
margin-safe), on ragged sizes, both block sizes these types take, both
drivers, padding canaries, distance-only and host-buffer solves."""
import numpy as np
import pytest

import graphgen
import oracle
from fwtest import check_pred_near_tight_f32, check_pred_tight_int, fw, gpu_solve, gpu_solve_dist_only

pytestmark = pytest.mark.gpu

INF64 = graphgen.INF_I64
PERSISTENT, PHASED = 1, 2


def _check_i64(W, D, P, Do, Po):
    np.testing.assert_array_equal(D, Do)
    check_pred_tight_int(W, Do, P, Po, inf=INF64)


def _f64_tol(Do, Po):
    reach = np.isfinite(Do)
    hops = oracle.hops(Po)
    tol = 1e-15 * np.maximum(hops, 1) * np.abs(Do)
    tol[~reach] = 0
    return tol


def _check_f64(W, D, P, Do, Po):
    reach = np.isfinite(Do)
    assert (np.isfinite(D) == reach).all(), "reachability differs"
    tol = _f64_tol(Do, Po)
    err = np.abs(D - Do)
    err[~reach] = 0
    assert (err <= tol).all(), "fp64 error above 1e-15 * hops at %d entries" % (err > tol).sum()
    return check_pred_near_tight_f32(W, Do, P, Po, tol)


@pytest.mark.parametrize("n", [1, 5, 33, 64, 100, 257, 600])
@pytest.mark.parametrize("bs", [32, 64])
@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
def test_i64(n, bs, driver):
    W = graphgen.dense_graph_i64(n, seed=n + bs, p=0.5, lo=1, hi=10 ** 12)
    Do, Po = oracle.fw_i64(W)
    D, P = gpu_solve(W, bs=bs, driver=driver, extra_ld=4)
    _check_i64(W, D, P, Do, Po)


@pytest.mark.parametrize("n", [1, 5, 33, 64, 100, 257, 600])
@pytest.mark.parametrize("bs", [32, 64])
@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
def test_f64(n, bs, driver):
    W = graphgen.dense_graph_f64(n, seed=n + bs + 1, p=0.5)
    Do, Po = oracle.fw_f64(W)
    D, P = gpu_solve(W, bs=bs, driver=driver, extra_ld=4)
    _check_f64(W, D, P, Do, Po)


@pytest.mark.parametrize("n", [300, 1000])
def test_f64_integer_weights_exact_and_drivers_agree(n):
    """Integer-valued fp64 weights: every sum is exact, so the distances are
    bit-exact, the predecessors tight, and the two drivers pick identical ones."""
    Wi = graphgen.dense_graph_i32(n, seed=7, p=0.4, lo=1, hi=20)
    W = np.where(Wi >= graphgen.INF_I32, np.inf, Wi.astype(np.float64))
    Do, Po = oracle.fw_f64(W)
    D1, P1 = gpu_solve(W, driver=PERSISTENT)
    D2, P2 = gpu_solve(W, driver=PHASED)
    np.testing.assert_array_equal(D1, Do)
    np.testing.assert_array_equal(D2, Do)
    np.testing.assert_array_equal(P1, P2)
    check_pred_near_tight_f32(W, Do, P1, Po, np.zeros_like(Do))


@pytest.mark.parametrize("kind", ["i64", "f64"])
def test_n4096_full_oracle(kind):
    """n = 4096, p = 0.5, automatic block size (64): the whole matrix."""
    n = 4096
    if kind == "i64":
        W = graphgen.dense_graph_i64(n, seed=2, p=0.5, lo=1, hi=10 ** 12)
        Do, Po = oracle.fw_i64(W)
        D, P = gpu_solve(W)
        _check_i64(W, D, P, Do, Po)
    else:
        W = graphgen.dense_graph_f64(n, seed=2, p=0.5)
        Do, Po = oracle.fw_f64(W)
        D, P = gpu_solve(W)
        differ = _check_f64(W, D, P, Do, Po)
        assert differ < 0.01 * n * n


@pytest.mark.parametrize("kind", ["i64", "f64"])
@pytest.mark.parametrize("driver", [PERSISTENT, PHASED])
def test_distance_only(kind, driver):
    n = 333
    if kind == "i64":
        W = graphgen.dense_graph_i64(n, seed=3, p=0.4, lo=1, hi=10 ** 9)
        Do, _ = oracle.fw_i64(W)
        D = gpu_solve_dist_only(W, driver=driver, extra_ld=4)
        np.testing.assert_array_equal(D, Do)
    else:
        W = graphgen.dense_graph_f64(n, seed=3, p=0.4)
        Do, Po = oracle.fw_f64(W)
        D = gpu_solve_dist_only(W, driver=driver, extra_ld=4)
        tol = _f64_tol(Do, Po)
        fin = np.isfinite(Do)
        assert (np.isfinite(D) == fin).all()
        assert (np.abs(D - Do)[fin] <= tol[fin]).all()


@pytest.mark.parametrize("kind", ["i64", "f64"])
def test_host_buffers(kind):
    m = fw()
    n = 500
    W = (graphgen.dense_graph_i64(n, seed=4, p=0.5, lo=1, hi=10 ** 12) if kind == "i64"
         else graphgen.dense_graph_f64(n, seed=4, p=0.5))
    ld = m.padded(n)
    Dh = np.zeros((n, ld), W.dtype)
    Dh[:, :n] = W
    Ph = np.zeros((n, ld), np.int32)
    m.fw_solve_host(Dh[:, :n], Ph[:, :n])
    if kind == "i64":
        Do, Po = oracle.fw_i64(W)
        _check_i64(W, Dh[:, :n], Ph[:, :n], Do, Po)
    else:
        Do, Po = oracle.fw_f64(W)
        _check_f64(W, Dh[:, :n], Ph[:, :n], Do, Po)


def test_wide_types_reject_what_they_do_not_support():
    import torch
    m = fw()
    n = 300
    D = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    P = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    with pytest.raises(m.FWError) as e:
        m.fw_solve_ex(D, P, m.Options.default(bs=128))
    assert e.value.code == 6
    with pytest.raises(m.FWError) as e:
        m.fw_solve_noalloc(D, P)
    assert e.value.code == 6
    with pytest.raises(m.FWError) as e:
        m.BatchedPlan([n], [n], m.FW_F64)
    assert e.value.code == 6


@pytest.mark.parametrize("dtype", ["i64", "f64"])
def test_peak_probe_wide(dtype):
    m = fw()
    rps, per_clk, mhz = m.fw_peak_probe(m.FW_I64 if dtype == "i64" else m.FW_F64)
    assert rps > 1e10 and per_clk > 0.1 and mhz > 100


def test_device_generator_wide_matches_host():
    import torch
    import graphgen.device as gdev
    n = 300
    t = torch.empty((n, n + 4), dtype=torch.int64, device="cuda")
    gdev.fill_i64(t[:, :n], seed=5, p=0.3, lo=1, hi=10 ** 12)
    np.testing.assert_array_equal(t[:, :n].cpu().numpy(),
                                  graphgen.dense_graph_i64(n, 5, 0.3, 1, 10 ** 12))
    f = torch.empty((n, n + 4), dtype=torch.float64, device="cuda")
    for kind in (0, 1):
        gdev.fill_f64(f[:, :n], seed=6, p=0.5, kind=kind)
        np.testing.assert_array_equal(f[:, :n].cpu().numpy(),
                                      graphgen.dense_graph_f64(n, 6, 0.5, kind=kind))
