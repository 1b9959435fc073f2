"""SSSP (Section 7.1.2, delta-stepping) on the weighted compressed graph:
distances equal the oracle's Dijkstra distances exactly (they are unique
integers), for every ID/offset mode that stores weights, with and without DM
relabeling, for several bucket widths, on small random graphs (every source)
and on a weighted R-MAT graph."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg

pytestmark = pytest.mark.gpu

MODES = [dict(id_mode=lg.LG_ID_GLOBAL, off_mode=lg.LG_OFF_PACKED),
         dict(id_mode=lg.LG_ID_GLOBAL, off_mode=lg.LG_OFF_EF),
         dict(id_mode=lg.LG_ID_GLOBAL, off_mode=lg.LG_OFF_EF, relabel=True),
         dict(id_mode=lg.LG_ID_CSR32),
         dict(id_mode=lg.LG_ID_CSR32, relabel=True)]


def dists(g, s, delta=0):
    return lg.lg_sssp(g, s, delta).cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("seed", range(4))
def test_sssp_small_graphs_every_source(seed):
    lg.load(auto_build=True)
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 60))
    edges = rng.integers(0, n, size=(int(rng.integers(0, 3 * n)), 2))
    h = gen.from_edges(n, edges, weighted=True, seed=seed + 7)
    for opts in MODES:
        g = lg.lg_encode(h.row_ptr, h.col, h.weights, **opts)
        for s in range(n):
            want = oracle.sssp(n, h.row_ptr, h.col, h.weights, s)
            assert np.array_equal(dists(g, s, delta=int(rng.integers(1, 300))), want), (opts, s)
        g.free()


@pytest.mark.parametrize("delta", [1, 16, 64, 255, 100000])
def test_sssp_rmat14_weighted(delta):
    lg.load(auto_build=True)
    h = gen.rmat(14, 16, seed=21, weighted=True)
    deg = h.degrees()
    srcs = [int(np.argmax(deg)), int(np.flatnonzero(deg)[5]), int(np.flatnonzero(deg)[-3])]
    isolated = np.flatnonzero(deg == 0)
    if isolated.size:
        srcs.append(int(isolated[0]))
    want = {s: oracle.sssp(h.n, h.row_ptr, h.col, h.weights, s) for s in srcs}
    for opts in MODES:
        g = lg.lg_encode(h.row_ptr, h.col, h.weights, **opts)
        for s in srcs:
            assert np.array_equal(dists(g, s, delta), want[s]), (opts, s)
        g.free()


def test_sssp_weights_at_fixed_width():
    """Weights stored at more bits than they need (omega = 12) decode the same."""
    lg.load(auto_build=True)
    h = gen.rmat(11, 8, seed=3, weighted=True)
    g = lg.lg_encode(h.row_ptr, h.col, h.weights, id_mode=lg.LG_ID_GLOBAL, off_mode=lg.LG_OFF_EF, weight_bits=12)
    assert g.stats()["omega"] == 12
    for s in (0, 100, 2047):
        assert np.array_equal(dists(g, s), oracle.sssp(h.n, h.row_ptr, h.col, h.weights, s))
    g.free()


def test_sssp_errors():
    lg.load(auto_build=True)
    h = gen.rmat(8, 4, seed=1)
    g = lg.lg_encode(h.row_ptr, h.col)  # no weights
    with pytest.raises(lg.LgError) as ei:
        lg.lg_sssp(g, 0)
    assert ei.value.status == 6
    g.free()
    hw = gen.rmat(8, 4, seed=1, weighted=True)
    g = lg.lg_encode(hw.row_ptr, hw.col, hw.weights)
    with pytest.raises(lg.LgError) as ei:
        lg.lg_sssp(g, hw.n)
    assert ei.value.status == 1
    g.free()
