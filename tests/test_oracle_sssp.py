"""Pins of the oracle's single-source shortest paths (Section 7.1.2 SSSP):
Floyd-Warshall brute force on small random weighted graphs, the closed form on
a weighted path, unit weights = BFS depths, and the defining properties
(no arc can shorten a distance; every reached vertex is reached by a tight
arc) on a weighted R-MAT graph."""
import numpy as np
import pytest

import gen
import oracle

INF64 = np.iinfo(np.uint64).max


def floyd_warshall(n, rp, col, w):
    big = np.iinfo(np.int64).max // 4
    d = np.full((n, n), big, dtype=np.int64)
    np.fill_diagonal(d, 0)
    for v in range(n):
        for j in range(int(rp[v]), int(rp[v + 1])):
            d[v, col[j]] = min(d[v, col[j]], int(w[j]))
    for k in range(n):
        d = np.minimum(d, d[:, [k]] + d[[k], :])
    return d, big


@pytest.mark.parametrize("seed", range(6))
def test_sssp_equals_floyd_warshall(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    m = int(rng.integers(0, 3 * n))
    edges = rng.integers(0, n, size=(m, 2))
    g = gen.from_edges(n, edges, weighted=True, seed=seed + 1)
    d, big = floyd_warshall(n, g.row_ptr, g.col, g.weights)
    for s in range(n):
        got = oracle.sssp(n, g.row_ptr, g.col, g.weights, s)
        want = np.where(d[s] >= big, INF64, d[s].astype(np.uint64))
        assert np.array_equal(got, want), (seed, s)


def test_sssp_weighted_path_closed_form():
    n = 50
    rng = np.random.default_rng(3)
    wts = rng.integers(1, 256, size=n - 1)
    # a path 0-1-...-49 with weight wts[i] on edge {i, i+1}, both arcs
    rp = np.zeros(n + 1, dtype=np.uint64)
    col, w = [], []
    for v in range(n):
        if v > 0:
            col.append(v - 1); w.append(wts[v - 1])
        if v + 1 < n:
            col.append(v + 1); w.append(wts[v])
        rp[v + 1] = len(col)
    col = np.array(col, dtype=np.uint32)
    w = np.array(w, dtype=np.uint32)
    got = oracle.sssp(n, rp, col, w, 0)
    assert np.array_equal(got, np.concatenate([[0], np.cumsum(wts)]).astype(np.uint64))
    got = oracle.sssp(n, rp, col, w, n - 1)
    assert np.array_equal(got, np.concatenate([np.cumsum(wts[::-1])[::-1], [0]]).astype(np.uint64))


def test_sssp_unit_weights_are_bfs_depths():
    g = gen.rmat(10, 8, seed=5)
    ones = np.ones(g.arcs, dtype=np.uint32)
    for s in (0, 17, int(np.argmax(g.degrees()))):
        dist = oracle.sssp(g.n, g.row_ptr, g.col, ones, s)
        depth = oracle.bfs(g.n, g.row_ptr, g.col, s)
        want = np.where(depth == np.iinfo(np.uint32).max, INF64, depth.astype(np.uint64))
        assert np.array_equal(dist, want)


def test_sssp_defining_properties_on_rmat():
    g = gen.rmat(12, 16, seed=9, weighted=True)
    deg = g.degrees()
    src = int(np.flatnonzero(deg)[7])
    dist = oracle.sssp(g.n, g.row_ptr, g.col, g.weights, src)
    u = np.repeat(np.arange(g.n), deg)
    v = g.col.astype(np.int64)
    reached_u = dist[u] != INF64
    # no arc shortens a distance
    assert np.all(dist[v][reached_u] <= dist[u][reached_u] + g.weights[reached_u])
    # an arc never leaves the reached set
    assert np.all((dist[u] == INF64) == (dist[v] == INF64))
    # every reached vertex but the source has a tight incoming arc
    tight = reached_u & (dist[u] + g.weights == dist[v])
    has_tight = np.zeros(g.n, dtype=bool)
    has_tight[v[tight]] = True
    reached = dist != INF64
    reached[src] = False
    assert np.all(has_tight[reached])
    assert dist[src] == 0
    # same reached set as BFS
    depth = oracle.bfs(g.n, g.row_ptr, g.col, src)
    assert np.array_equal(dist != INF64, depth != np.iinfo(np.uint32).max)


def test_sssp_rejects_bad_source():
    g = gen.from_edges(3, [(0, 1)], weighted=True)
    with pytest.raises(oracle.OracleError):
        oracle.sssp(3, g.row_ptr, g.col, g.weights, 3)
