"""The greedy relabeling heuristic (Section 3.2.2, Listing 1) on the GPU:
permutation, streams and offsets byte-equal to the oracle's, decoded
neighborhoods equal to the input rows (original IDs), BFS and PageRank equal
to the oracle's on the original graph, in every mode, including weights."""
import itertools

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg
from helpers import all_graphs
from test_gpu_parity import (OFFS, MODES, assert_arrays_equal, assert_bfs, assert_neighbors, assert_pagerank, dev,
                             encode_both)

pytestmark = pytest.mark.gpu
GREEDY = lg.LG_RELABEL_GREEDY


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lg.load(auto_build=True)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_greedy_tiny_graphs(n):
    for edges in all_graphs(n):
        h = gen.from_edges(n, edges) if edges else gen.from_edges(n, np.zeros((0, 2)))
        for mode, off in itertools.product(range(3), range(2)):
            g, e = encode_both(n, h.row_ptr, h.col, mode=mode, off=off, relabel=GREEDY)
            assert_arrays_equal(g, e)
            assert_neighbors(g, h.row_ptr, h.col, n)
            g.free()


@pytest.mark.parametrize("mode,off", list(itertools.product(range(3), range(2))))
def test_greedy_rmat16(mode, off):
    h = gen.rmat_s16_ef16()
    g, e = encode_both(h.n, h.row_ptr, h.col, mode=mode, off=off, relabel=GREEDY)
    assert_arrays_equal(g, e)
    assert_neighbors(g, h.row_ptr, h.col, h.n)
    deg = h.degrees()
    assert_bfs(g, h.n, h.row_ptr, h.col, [int(np.argmax(deg)), int(np.flatnonzero(deg)[9]), 0])
    assert_pagerank(g, h.n, h.row_ptr, h.col, iters=10)
    g.free()


def test_greedy_community_and_widths():
    """On a community graph the greedy labels shrink the local widths (the
    heuristic's purpose); the streams stay byte-equal to the oracle's."""
    h = gen.community(log2n=16, log2block=10, seed=2)
    bits = {}
    for relabel in (lg.LG_RELABEL_NONE, lg.LG_RELABEL_DM, GREEDY):
        g, e = encode_both(h.n, h.row_ptr, h.col, mode=1, off=1, relabel=relabel)
        assert_arrays_equal(g, e)
        bits[relabel] = lg.lg_stats_get(g)["bits_A"]
        g.free()
    assert bits[GREEDY] < bits[lg.LG_RELABEL_NONE]


def test_greedy_weighted_and_sssp():
    h = gen.rmat(12, 8, seed=8, weighted=True)
    g, e = encode_both(h.n, h.row_ptr, h.col, h.weights, mode=0, off=1, relabel=GREEDY)
    assert_arrays_equal(g, e)
    assert_neighbors(g, h.row_ptr, h.col, h.n, w=h.weights)
    for s in (0, 77, int(np.argmax(h.degrees()))):
        d = lg.lg_sssp(g, s).cpu().numpy().view(np.uint64)
        assert np.array_equal(d, oracle.sssp(h.n, h.row_ptr, h.col, h.weights, s))
    g.free()


def test_bad_relabel_value():
    h = gen.rmat(6, 4, seed=1)
    with pytest.raises(lg.LgError) as ei:
        lg.lg_encode(dev(h.row_ptr, np.int64), dev(h.col, np.int32), relabel=3)
    assert ei.value.status == 1
