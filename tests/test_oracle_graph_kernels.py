"""Pins of the oracle's BFS and PageRank.

BFS: brute force (Floyd-Warshall over the adjacency matrix) on small graphs,
and path / star / disconnected special cases.
PageRank: exact 1/n on regular graphs, the closed two-state recurrence of a
star, the sum rule, the fixed point of (I - d A D^-1) r = (1-d)/n solved
directly, the same for the personalized form, and isolated vertices.
"""
import numpy as np
import pytest

import gen
import oracle
from helpers import csr_from_edges

INF = np.iinfo(np.uint32).max


def _adj(n, rp, col):
    A = np.zeros((n, n))
    for v in range(n):
        A[v, col[rp[v]:rp[v + 1]]] = 1
    return A


@pytest.mark.parametrize("seed", range(6))
def test_bfs_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(0, 2 * n))
    rp, col, _ = csr_from_edges(n, rng.integers(0, n, size=(m, 2)).tolist())
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    A = _adj(n, rp, col)
    D[A > 0] = 1
    for k in range(n):
        D = np.minimum(D, D[:, [k]] + D[[k], :])
    for s in range(n):
        got = oracle.bfs(n, rp, col, s)
        want = np.where(np.isinf(D[s]), INF, D[s]).astype(np.uint32)
        assert np.array_equal(got, want)


def test_bfs_special_cases():
    n = 50
    rp, col, _ = csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    assert np.array_equal(oracle.bfs(n, rp, col, 0), np.arange(n, dtype=np.uint32))
    rp, col, _ = csr_from_edges(n, [(0, i) for i in range(1, n)])
    d = oracle.bfs(n, rp, col, 3)
    assert d[3] == 0 and d[0] == 1 and set(d.tolist()) == {0, 1, 2}
    rp, col, _ = csr_from_edges(6, [(0, 1), (2, 3)])
    d = oracle.bfs(6, rp, col, 0)
    assert d.tolist() == [0, 1, INF, INF, INF, INF]


@pytest.mark.parametrize("n", [5, 12])
def test_pagerank_regular_is_uniform(n):
    # cycle (2-regular) and complete graph: r_t = 1/n for every t
    for edges in ([(i, (i + 1) % n) for i in range(n)],
                  [(i, j) for i in range(n) for j in range(i + 1, n)]):
        rp, col, _ = csr_from_edges(n, edges)
        r = oracle.pagerank(n, rp, col, 0.85, 7)
        assert np.allclose(r, 1.0 / n, rtol=0, atol=1e-15)


def test_pagerank_star_recurrence():
    k, d, T = 9, 0.85, 12
    n = k + 1
    rp, col, _ = csr_from_edges(n, [(0, i) for i in range(1, n)])
    r = oracle.pagerank(n, rp, col, d, T)
    h = l = 1.0 / n
    for _ in range(T):  # hub gets k leaves of degree 1; a leaf gets hub / k
        h, l = (1 - d) / n + d * k * l, (1 - d) / n + d * h / k
    assert abs(r[0] - h) < 1e-15 and np.allclose(r[1:], l, rtol=0, atol=1e-15)


def test_pagerank_sum_rule_and_fixed_point():
    g = gen.rmat(6, 4, seed=11)
    n, rp, col = g.n, g.row_ptr, g.col
    deg = g.degrees()
    keep = deg > 0
    d = 0.85
    r = oracle.pagerank(n, rp, col, d, 300)
    A = _adj(n, rp, col)
    M = A / np.where(deg > 0, deg, 1)[None, :]  # M[v, u] = [u in N_v] / d_u
    want = np.linalg.solve(np.eye(n) - d * M, np.full(n, (1 - d) / n))
    assert np.allclose(r, want, rtol=1e-10, atol=0)
    # isolated vertices keep (1 - d)/n; the rest sum to 1 - (#isolated)(1-d)/n ... exactly per step
    assert np.allclose(r[~keep], (1 - d) / n)
    r3 = oracle.pagerank(n, rp, col, d, 3)
    if keep.all():
        assert abs(r3.sum() - 1.0) < 1e-12


def test_pagerank_sum_rule_connected():
    n = 40
    rng = np.random.default_rng(3)
    edges = [(i, i + 1) for i in range(n - 1)] + rng.integers(0, n, size=(60, 2)).tolist()
    rp, col, _ = csr_from_edges(n, edges)
    for T in (1, 2, 5, 20):
        assert abs(oracle.pagerank(n, rp, col, 0.85, T).sum() - 1.0) < 1e-12


def test_personalized_pagerank_fixed_point():
    n = 30
    rng = np.random.default_rng(4)
    edges = [(i, i + 1) for i in range(n - 1)] + rng.integers(0, n, size=(40, 2)).tolist()
    rp, col, _ = csr_from_edges(n, edges)
    d, s = 0.85, 7
    A = _adj(n, rp, col)
    deg = A.sum(axis=0)
    M = A / deg[None, :]
    e = np.zeros(n)
    e[s] = 1
    want = np.linalg.solve(np.eye(n) - d * M, (1 - d) * e)
    r = oracle.pagerank(n, rp, col, d, 400, personalize=s)
    assert np.allclose(r, want, rtol=1e-10, atol=1e-14)
    r1 = oracle.pagerank(n, rp, col, d, 1, personalize=s)
    nb = col[rp[s]:rp[s + 1]]
    assert r1[s] == pytest.approx(1 - d)
    assert np.allclose(r1[nb], d / deg[s])
