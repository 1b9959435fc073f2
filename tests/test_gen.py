"""Properties of the seeded input generators (inputs only, no method arithmetic)."""
import numpy as np

import gen


def _check_simple_symmetric(g):
    rp, col = g.row_ptr, g.col
    assert rp[0] == 0 and rp[-1] == g.arcs and np.all(np.diff(rp.astype(np.int64)) >= 0)
    src = np.repeat(np.arange(g.n, dtype=np.uint64), np.diff(rp).astype(np.int64))
    assert np.all(col < g.n)
    assert not np.any(src == col), "self loop"
    key = src * np.uint64(g.n) + col
    assert np.all(np.diff(key.astype(np.int64)) > 0), "rows not strictly increasing"
    rkey = np.sort(col.astype(np.uint64) * np.uint64(g.n) + src)
    assert np.array_equal(np.sort(key), rkey), "not symmetric"


def test_rmat_properties_and_determinism():
    g = gen.rmat(10, 8, seed=3)
    _check_simple_symmetric(g)
    h = gen.rmat(10, 8, seed=3, threads=1)
    assert np.array_equal(g.row_ptr, h.row_ptr) and np.array_equal(g.col, h.col)
    k = gen.rmat(10, 8, seed=4)
    assert not np.array_equal(g.col, k.col[: g.arcs]) or g.arcs != k.arcs


def test_rmat_weights_symmetric_in_range():
    g = gen.rmat(9, 8, seed=5, weighted=True)
    w = g.weights
    assert w.min() >= 1 and w.max() <= 255
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    d = {(int(a), int(b)): int(x) for a, b, x in zip(src, g.col, w)}
    assert all(d[(b, a)] == x for (a, b), x in d.items())


def test_community_properties():
    g = gen.community(log2n=14, log2block=10, seed=2)
    _check_simple_symmetric(g)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    # most arcs stay inside the block before the global permutation
    h = gen.community(log2n=14, log2block=10, seed=2, permute=False)
    hs = np.repeat(np.arange(h.n), np.diff(h.row_ptr).astype(np.int64))
    intra = np.mean((hs >> 10) == (h.col.astype(np.int64) >> 10))
    assert intra > 0.85
    assert 15 < g.arcs / g.n < 30
    assert len(src) == g.arcs


def test_sources_distinct_nonzero_degree():
    g = gen.rmat(8, 2, seed=1)
    s = gen.sources(g, 16, seed=9)
    assert len(set(s.tolist())) == 16
    assert np.all(g.degrees()[s] > 0)
