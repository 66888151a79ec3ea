"""The shared seeded input generator: determinism, ranges and row slicing (CPU)."""
import numpy as np

import graphgen


def test_splitmix_reference_values():
    # SplitMix64 stream from state 0 (the generator's published test sequence
    # starts 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F).
    ks = np.arange(3, dtype=np.uint64)
    with np.errstate(over="ignore"):
        states = ks * graphgen.GAMMA
    outs = [int(x) for x in graphgen.splitmix64(states)]
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_int_graph_ranges_and_density():
    n = 300
    W = graphgen.dense_graph_i32(n, seed=3, p=0.3, lo=1, hi=100)
    off = ~np.eye(n, dtype=bool)
    e = W[off] < graphgen.INF_I32
    assert abs(e.mean() - 0.3) < 0.01
    assert W[off][e].min() >= 1 and W[off][e].max() <= 100
    assert (np.diag(W) == 0).all()
    np.testing.assert_array_equal(W, graphgen.dense_graph_i32(n, seed=3, p=0.3, lo=1, hi=100,
                                                              chunk_rows=7))
    rows = np.array([0, 5, 299])
    np.testing.assert_array_equal(W[rows], graphgen.dense_graph_i32(n, 3, 0.3, 1, 100, rows=rows))


def test_float_graph_ranges():
    n = 200
    W = graphgen.dense_graph_f32(n, seed=4, p=0.5)
    off = ~np.eye(n, dtype=bool)
    fin = np.isfinite(W[off])
    assert abs(fin.mean() - 0.5) < 0.02
    assert W[off][fin].min() > 0 and W[off][fin].max() <= 1
    V = graphgen.dense_graph_f32(n, seed=4, p=0.5, kind=graphgen.KIND_ONE_TWO)
    assert V[off][np.isfinite(V[off])].min() >= 1 and V[off][np.isfinite(V[off])].max() <= 2


def test_batch_sizes_and_normals():
    ns = graphgen.batch_sizes(7, 512)
    assert ns.min() >= 64 and ns.max() <= 2048 and len(set(ns.tolist())) > 300
    z = graphgen.normal_f32((100000,), seed=1)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.02


def test_wide_graph_ranges_and_exactness():
    n = 200
    W = graphgen.dense_graph_i64(n, seed=5, p=0.4, lo=1, hi=10 ** 12)
    off = ~np.eye(n, dtype=bool)
    e = W[off] < graphgen.INF_I64
    assert abs(e.mean() - 0.4) < 0.02
    assert W[off][e].min() >= 1 and W[off][e].max() <= 10 ** 12
    assert W[off][e].max() > 2 ** 31  # beyond the int32 range
    assert (np.diag(W) == 0).all() and W.dtype == np.int64
    # the same counters as the int32 generator: same edges, same draws mod span
    W32 = graphgen.dense_graph_i32(n, seed=5, p=0.4, lo=1, hi=100)
    np.testing.assert_array_equal(W32[off] < graphgen.INF_I32, e)
    V = graphgen.dense_graph_f64(n, seed=6, p=0.5)
    fin = np.isfinite(V[off])
    assert V[off][fin].min() > 0 and V[off][fin].max() <= 1
    # full 53-bit mantissas: most weights are not representable in fp32
    assert (V[off][fin].astype(np.float32).astype(np.float64) != V[off][fin]).mean() > 0.99
    U = graphgen.dense_graph_f64(n, seed=6, p=0.5, kind=graphgen.KIND_ONE_TWO)
    u = U[off][np.isfinite(U[off])]
    assert u.min() >= 1 and u.max() < 2
    np.testing.assert_array_equal(V, graphgen.dense_graph_f64(n, 6, 0.5, chunk_rows=13))
