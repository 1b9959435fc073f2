"""Pins of the oracle's greedy relabeling heuristic (Section 3.2.2, Listing 1,
read with 0-based labels, every sorted vertex visited, leftovers in ID order):
a hand-worked example, an independent formulation (a vertex's label is the
rank of its first appearance in the neighbor lists taken by increasing degree;
vertices that never appear follow in ID order), and round trips through every
encoding mode."""
import os

import numpy as np
import pytest

import gen
import oracle
from helpers import parse_golden

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "greedy_relabel.txt")


def read_golden():
    fx = parse_golden(GOLDEN)
    return fx["graph"]["n"], fx["graph"]["edges"], np.array(fx["greedy_relabel"]["perm"], dtype=np.uint32)


def first_appearance_perm(n, rp, col):
    deg = np.diff(rp).astype(np.int64)
    order = np.lexsort((np.arange(n), deg))  # degree ascending, then ID
    seq = np.concatenate([col[rp[v]:rp[v + 1]] for v in order]) if rp[-1] else np.zeros(0, np.uint32)
    first = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(first, seq.astype(np.int64), np.arange(seq.size))
    new_order = np.lexsort((np.arange(n), first))
    perm = np.empty(n, dtype=np.uint32)
    perm[new_order] = np.arange(n, dtype=np.uint32)
    return perm


def test_greedy_relabel_golden():
    n, edges, want = read_golden()
    g = gen.from_edges(n, edges)
    e = oracle.encode(n, g.row_ptr, g.col, id_mode=oracle.ID_LOCAL, relabel=oracle.RELABEL_GREEDY)
    assert np.array_equal(e.perm, want)
    assert np.array_equal(e.inv_perm[want], np.arange(n, dtype=np.uint32))


@pytest.mark.parametrize("seed", range(8))
def test_greedy_relabel_first_appearance(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    edges = rng.integers(0, n, size=(int(rng.integers(0, 4 * n)), 2))
    g = gen.from_edges(n, edges)
    e = oracle.encode(n, g.row_ptr, g.col, id_mode=oracle.ID_LOCAL_GAP, relabel=oracle.RELABEL_GREEDY)
    assert np.array_equal(e.perm, first_appearance_perm(n, g.row_ptr, g.col))
    # the first vertex with neighbors hands out labels 0..d-1 in row order
    deg = np.diff(g.row_ptr)
    if deg.sum():
        order = np.lexsort((np.arange(n), deg))
        v = order[np.flatnonzero(deg[order] > 0)[0]]
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert np.array_equal(e.perm[nb], np.arange(nb.size, dtype=np.uint32))


def test_greedy_relabel_on_rmat():
    g = gen.rmat(11, 8, seed=4)
    e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=oracle.ID_LOCAL, relabel=oracle.RELABEL_GREEDY)
    assert np.array_equal(e.perm, first_appearance_perm(g.n, g.row_ptr, g.col))
    assert np.array_equal(np.sort(e.perm), np.arange(g.n, dtype=np.uint32))


@pytest.mark.parametrize("id_mode", [oracle.ID_GLOBAL, oracle.ID_LOCAL, oracle.ID_LOCAL_GAP])
@pytest.mark.parametrize("off_mode", [oracle.OFF_PACKED, oracle.OFF_EF])
def test_greedy_relabel_round_trip(id_mode, off_mode):
    g = gen.rmat(9, 8, seed=6)
    e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=id_mode, off_mode=off_mode, relabel=oracle.RELABEL_GREEDY)
    for v in range(0, g.n, 7):
        assert np.array_equal(e.neighbors(v), g.col[g.row_ptr[v]:g.row_ptr[v + 1]])
