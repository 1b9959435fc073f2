"""Full-size parity on the benchmark workload, in the launch configuration
bench.py times: the community graph with 2^24 vertices (392,627,612 arcs),
DM relabel + local-gap IDs + Elias-Fano offsets (select samples every 512),
BFS from the same 16 seeded sources, 20 PageRank iterations (d = 0.85).

Compared with the oracle: the whole A stream, the Elias-Fano arrays and the
permutation byte for byte; the whole-graph decode (row offsets in full, 20,000
stored rows); 20,000 sampled neighborhoods; all 16 BFS depth rows; every
PageRank value within 1e-4 relative.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg

pytestmark = pytest.mark.gpu

PR_RTOL = 1e-4


@pytest.fixture(scope="module")
def oracle_ranks(community):
    g0, _ = community
    return oracle.pagerank(g0.n, g0.row_ptr, g0.col, 0.85, 20, threads=16)


@pytest.fixture(scope="module")
def community():
    lg.load(auto_build=True)
    g0 = gen.community_2p24(seed=2)
    rp = torch.from_numpy(g0.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy(g0.col.view(np.int32)).cuda()
    g = lg.lg_encode(rp, col, id_mode=lg.LG_ID_LOCAL_GAP, off_mode=lg.LG_OFF_EF, relabel=True, select_sample=512)
    yield g0, g
    g.free()


@pytest.fixture(scope="module")
def oracle_encoded(community):
    g0, _ = community
    return oracle.encode(g0.n, g0.row_ptr, g0.col, id_mode=oracle.ID_LOCAL_GAP, off_mode=oracle.OFF_EF,
                         relabel=True, sample=512)


def test_fullsize_streams_byte_equal(community, oracle_encoded):
    g0, g = community
    e = oracle_encoded
    a = lg.lg_arrays_get(g)
    st = lg.lg_stats_get(g)
    assert st["bits_A"] == e.bits_A and st["ef_l"] == e.ef_l
    assert np.array_equal(a["perm"], e.perm) and np.array_equal(a["inv_perm"], e.inv_perm)
    assert np.array_equal(a["ef_low"], e.ef_low)
    assert np.array_equal(a["ef_high"], e.ef_high)
    assert np.array_equal(a["ef_samples"], e.samples)
    assert np.array_equal(a["A"], e.A)
    # bytes: compressed payload against the 32-bit CSR of the same graph
    assert (st["bits_A"] + st["bits_O"]) / 8 < 0.75 * (4 * g0.arcs + 8 * (g0.n + 1))


def test_fullsize_whole_graph_decode(community, oracle_encoded):
    """lg_decode of the whole graph (stored order, stored labels): row offsets
    in full from the relabeled degrees, rows of 20,000 stored vertices (the
    hub tiles first) against the oracle's bit-by-bit decode."""
    g0, g = community
    e = oracle_encoded
    rp, col = lg.lg_decode(g)
    rp = rp.cpu().numpy().view(np.uint64)
    col = col.cpu().numpy().view(np.uint32)
    sdeg = np.empty(g0.n, dtype=np.uint64)
    sdeg[e.perm] = np.diff(g0.row_ptr)
    want = np.zeros(g0.n + 1, dtype=np.uint64)
    np.cumsum(sdeg, out=want[1:])
    assert np.array_equal(rp, want)
    rng = np.random.default_rng(13)
    vs = np.concatenate([np.arange(2048), np.arange(g0.n - 1024, g0.n), rng.integers(0, g0.n, size=16928)])
    for v in vs:
        assert np.array_equal(col[rp[v]:rp[v + 1]], e.decode_raw(int(v))), f"stored vertex {v}"


def test_fullsize_sampled_neighborhoods(community):
    g0, g = community
    rng = np.random.default_rng(11)
    vs = rng.integers(0, g0.n, size=20000).astype(np.uint32)
    vs[:10] = np.argsort(-g0.degrees())[:10]  # the hubs
    off, ids = lg.lg_neighbors(g, torch.from_numpy(vs.view(np.int32)).cuda())
    off = off.cpu().numpy().view(np.uint64)
    ids = ids.cpu().numpy().view(np.uint32)
    for i, v in enumerate(vs):
        assert np.array_equal(ids[off[i]:off[i + 1]], g0.col[g0.row_ptr[v]:g0.row_ptr[v + 1]])


def test_fullsize_bfs_16_sources(community):
    g0, g = community
    src = gen.sources(g0, 16, seed=7)  # the bench's sources
    d = lg.lg_bfs(g, torch.from_numpy(src.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    with ThreadPoolExecutor(8) as ex:  # the oracle runs one BFS per thread
        want = list(ex.map(lambda s: oracle.bfs(g0.n, g0.row_ptr, g0.col, int(s)), src))
    for i, s in enumerate(src):
        assert np.array_equal(d[i], want[i]), f"source {s}"


def test_fullsize_pagerank_20(community, oracle_ranks):
    g0, g = community
    r = lg.lg_pagerank(g, 0.85, 20).cpu().numpy().astype(np.float64)
    want = oracle_ranks
    rel = np.abs(r - want) / want
    assert rel.max() <= PR_RTOL, f"max rel err {rel.max():.3e}"


def test_fullsize_csr32_baseline_pagerank(community, oracle_ranks):
    g0, _ = community
    rp = torch.from_numpy(g0.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy(g0.col.view(np.int32)).cuda()
    g = lg.lg_encode(rp, col, id_mode=lg.LG_ID_CSR32)
    r = lg.lg_pagerank(g, 0.85, 20).cpu().numpy().astype(np.float64)
    assert (np.abs(r - oracle_ranks) / oracle_ranks).max() <= PR_RTOL
