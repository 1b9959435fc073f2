"""Full-size parity on the largest configuration: R-MAT scale 27 (134,217,728
vertices, edge factor 16, ~4.29e9 stored arcs), integer weights in [1, 255]
stored at 8 bits, global 27-bit IDs, Elias-Fano offsets -- 35-bit records and
bit positions far past 2^32.  The graph is built on the device by the seeded
generator (the same edges as the host generator) and copied to the host for
the oracle.

The oracle cannot re-encode 1.5e11 bits one at a time within a test, so it is
compared on what it can compute piece by piece: the whole Elias-Fano offset
structure, 200 windows of the A stream (first, last and random), 4,000 sampled
neighborhoods with weights, two of the 16 BFS sources in full (all 16 checked
for the properties every BFS depth array has), PageRank after 3 iterations in
full (after 20, the sum rule), and SSSP over the 8-bit weights from one source
in full (Dijkstra) and from three more by the defining properties.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg

pytestmark = pytest.mark.gpu

INF = np.iinfo(np.uint32).max


@pytest.fixture(scope="module")
def rmat27():
    lg.load(auto_build=True)
    rp, col, w = gen.rmat_gpu(27, 16, seed=5, weighted=True)
    g = lg.lg_encode(rp, col, w, id_mode=lg.LG_ID_GLOBAL, off_mode=lg.LG_OFF_EF, weight_bits=8)
    host = (rp.cpu().numpy().view(np.uint64), col.cpu().numpy().view(np.uint32), w.cpu().numpy().view(np.uint32))
    del rp, col, w
    torch.cuda.empty_cache()
    yield g, host
    g.free()


def test_rmat27_widths_and_offsets(rmat27):
    g, (rp, col, w) = rmat27
    n, arcs = rp.shape[0] - 1, col.shape[0]
    st = lg.lg_stats_get(g)
    assert n == 1 << 27 and arcs > 4_000_000_000
    assert st["s"] == 27 and st["omega"] == 8 and st["bits_A"] == arcs * 35
    low, high, smp, l = oracle.ef_build(rp, sample=512)
    a = lg.lg_arrays_get(g)
    assert st["ef_l"] == l
    assert np.array_equal(a["ef_low"], low) and np.array_equal(a["ef_high"], high)
    assert np.array_equal(a["ef_samples"], smp)
    used = (st["bits_A"] + 63) // 64
    rng = np.random.default_rng(27)
    starts = [0, used - 64] + rng.integers(0, used - 64, size=198).tolist()
    for w0 in starts:
        want = oracle.global_words(col, w, 27, 8, int(w0), int(w0) + 64)
        assert np.array_equal(a["A"][w0:w0 + 64], want), f"A words at {w0}"
    assert not np.any(a["A"][used:])


def test_rmat27_sampled_neighborhoods(rmat27):
    g, (rp, col, w) = rmat27
    n = rp.shape[0] - 1
    rng = np.random.default_rng(5)
    deg = np.diff(rp)
    vs = np.concatenate([np.argsort(-deg)[:8], rng.integers(0, n, size=3992)]).astype(np.uint32)
    off, ids, wts = lg.lg_neighbors(g, torch.from_numpy(vs.view(np.int32)).cuda(), with_weights=True)
    off = off.cpu().numpy().view(np.uint64)
    ids = ids.cpu().numpy().view(np.uint32)
    wts = wts.cpu().numpy().view(np.uint32)
    for i, v in enumerate(vs):
        lo, hi = rp[v], rp[v + 1]
        assert np.array_equal(ids[off[i]:off[i + 1]], col[lo:hi])
        assert np.array_equal(wts[off[i]:off[i + 1]], w[lo:hi])


def test_rmat27_bfs_16_sources(rmat27):
    g, (rp, col, _) = rmat27
    n = rp.shape[0] - 1

    class G:  # sources() needs only n and row_ptr
        pass

    G.n, G.row_ptr = n, rp
    src = gen.sources(G, 16, seed=7)
    d = lg.lg_bfs(g, torch.from_numpy(src.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    for i in (0, 9):
        assert np.array_equal(d[i], oracle.bfs(n, rp, col, int(src[i]))), f"source {src[i]}"
    rng = np.random.default_rng(1)
    arcs_s = rng.integers(0, col.shape[0], size=2_000_000)
    us = np.searchsorted(rp, arcs_s, side="right") - 1
    vs = col[arcs_s]
    for i, s in enumerate(src):
        row = d[i]
        assert row[s] == 0
        du, dv = row[us].astype(np.int64), row[vs].astype(np.int64)
        both = (du != INF) & (dv != INF)
        assert np.all(np.abs(du[both] - dv[both]) <= 1)
        assert np.all((du == INF) == (dv == INF))  # an arc never leaves a component


def test_rmat27_pagerank(rmat27):
    g, (rp, col, _) = rmat27
    n = rp.shape[0] - 1
    r3 = lg.lg_pagerank(g, 0.85, 3).cpu().numpy().astype(np.float64)
    want = oracle.pagerank(n, rp, col, 0.85, 3, threads=16)
    nz = want > 0
    assert (np.abs(r3[nz] - want[nz]) / want[nz]).max() <= 1e-4
    r20 = lg.lg_pagerank(g, 0.85, 20).cpu().numpy().astype(np.float64)
    isolated = int((np.diff(rp) == 0).sum())
    assert abs(r20.sum() - (1.0 - isolated * 0.85 / n)) < 1e-3
    assert r20.min() >= (1 - 0.85) / n * (1 - 1e-5)


def test_rmat27_sssp(rmat27):
    g, (rp, col, w) = rmat27
    n = rp.shape[0] - 1
    deg = np.diff(rp)
    nz = np.flatnonzero(deg)
    srcs = [int(nz[12345]), int(np.argmax(deg)), int(nz[-7]), int(nz[len(nz) // 2])]
    d0 = lg.lg_sssp(g, srcs[0]).cpu().numpy().view(np.uint64)
    assert np.array_equal(d0, oracle.sssp(n, rp, col, w, srcs[0]))
    rng = np.random.default_rng(2)
    arcs_s = rng.integers(0, col.shape[0], size=3_000_000)
    us = np.searchsorted(rp, arcs_s, side="right") - 1
    vs = col[arcs_s]
    ws = w[arcs_s].astype(np.uint64)
    INF64 = np.iinfo(np.uint64).max
    for s in srcs[1:]:
        d = lg.lg_sssp(g, s).cpu().numpy().view(np.uint64)
        assert d[s] == 0
        du, dv = d[us], d[vs]
        reach = du != INF64
        assert np.all((du == INF64) == (dv == INF64))
        assert np.all(dv[reach] <= du[reach] + ws[reach])  # no arc shortens a distance
        depth = oracle.bfs(n, rp, col, s) if s == srcs[1] else None
        if depth is not None:
            assert np.array_equal(d != INF64, depth != INF)
