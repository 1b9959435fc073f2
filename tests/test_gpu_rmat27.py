"""Full-size parity on the largest configuration: R-MAT scale 27 (134,217,728
vertices, edge factor 16, ~4.22e9 stored arcs), integer weights in [1, 255]
stored at 8 bits, global 27-bit IDs, Elias-Fano offsets -- 35-bit records and
bit positions far past 2^32.  The graph is built on the device by the seeded
generator (the same edges as the host generator) and copied to the host for
the oracle.

Compared with the oracle in full: the whole Elias-Fano offset structure, the
whole A stream (1.48e11 bits, window by window with the oracle's bit-by-bit
encoder on every host core), all 16 BFS depth rows, every PageRank value after
20 iterations (1e-4 relative), SSSP over the 8-bit weights from one source
(Dijkstra; three more sources by the defining properties); the whole-graph
decode against the input CSR; 4,000 sampled neighborhoods with weights.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg

pytestmark = pytest.mark.gpu

INF = np.iinfo(np.uint32).max
NPROC = len(os.sched_getaffinity(0))


@pytest.fixture(scope="module")
def rmat27():
    lg.load(auto_build=True)
    rp, col, w = gen.rmat_gpu(27, 16, seed=5, weighted=True)
    g = lg.lg_encode(rp, col, w, id_mode=lg.LG_ID_GLOBAL, off_mode=lg.LG_OFF_EF, weight_bits=8)
    host = (rp.cpu().numpy().view(np.uint64), col.cpu().numpy().view(np.uint32), w.cpu().numpy().view(np.uint32))
    yield g, host, (rp, col, w)
    g.free()


def _sources(n, rp):
    class G:  # sources() needs only n and row_ptr
        pass

    G.n, G.row_ptr = n, rp
    return gen.sources(G, 16, seed=7)


def test_rmat27_widths_and_offsets(rmat27):
    g, (rp, col, w), _ = rmat27
    n, arcs = rp.shape[0] - 1, col.shape[0]
    st = lg.lg_stats_get(g)
    assert n == 1 << 27 and arcs > 4_000_000_000
    assert st["s"] == 27 and st["omega"] == 8 and st["bits_A"] == arcs * 35
    low, high, smp, l = oracle.ef_build(rp, sample=512)
    ef = lg.lg_arrays_device(g)
    assert st["ef_l"] == l
    assert np.array_equal(ef["ef_low"].cpu().numpy().view(np.uint64), low)
    assert np.array_equal(ef["ef_high"].cpu().numpy().view(np.uint64), high)
    assert np.array_equal(ef["ef_samples"].cpu().numpy().view(np.uint64), smp)


def test_rmat27_whole_A_stream(rmat27):
    """Every word of the A stream equals the oracle's bit-by-bit encoding
    (Sections 3.2.1 and 3.3: 27-bit IDs, each followed by its 8-bit weight);
    the padding and guard words are zero."""
    g, (rp, col, w), _ = rmat27
    st = lg.lg_stats_get(g)
    A = lg.lg_arrays_device(g)["A"]
    used = (st["bits_A"] + 63) // 64
    W = 1 << 24
    wins = [(w0, min(w0 + W, used)) for w0 in range(0, used, W)]
    torch.cuda.synchronize()
    with ThreadPoolExecutor(NPROC) as ex:
        for b in range(0, len(wins), NPROC):
            batch = wins[b:b + NPROC]
            futs = [ex.submit(oracle.global_words, col, w, 27, 8, w0, w1) for w0, w1 in batch]
            for (w0, w1), f in zip(batch, futs):
                got = A[w0:w1].cpu().numpy().view(np.uint64)
                assert np.array_equal(got, f.result()), f"A words [{w0}, {w1})"
    assert not torch.any(A[used:]).item()


def test_rmat27_whole_graph_decode(rmat27):
    """lg_decode of a graph with global IDs and no relabel is the input CSR
    itself, weights included."""
    g, _, (rp_d, col_d, w_d) = rmat27
    rp, col, wt = lg.lg_decode(g, with_weights=True)
    assert torch.equal(rp, rp_d)
    assert torch.equal(col, col_d)
    assert torch.equal(wt, w_d)
    del rp, col, wt
    torch.cuda.empty_cache()


def test_rmat27_sampled_neighborhoods(rmat27):
    g, (rp, col, w), _ = rmat27
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
    """All 16 depth rows equal the oracle's FIFO BFS on the input CSR."""
    g, (rp, col, _), _ = rmat27
    n = rp.shape[0] - 1
    src = _sources(n, rp)
    d = lg.lg_bfs(g, torch.from_numpy(src.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    with ThreadPoolExecutor(min(16, NPROC)) as ex:  # the oracle runs one BFS per thread
        want = ex.map(lambda s: oracle.bfs(n, rp, col, int(s)), src)
        for i, wd in enumerate(want):
            assert np.array_equal(d[i], wd), f"source {src[i]}"


def test_rmat27_pagerank_20(rmat27):
    """Every vertex within 1e-4 relative of the FP64 oracle after the 20
    iterations the workload runs."""
    g, (rp, col, _), _ = rmat27
    n = rp.shape[0] - 1
    r = lg.lg_pagerank(g, 0.85, 20).cpu().numpy().astype(np.float64)
    want = oracle.pagerank(n, rp, col, 0.85, 20, threads=NPROC)
    nz = want > 0
    rel = np.abs(r[nz] - want[nz]) / want[nz]
    assert rel.max() <= 1e-4, f"max rel err {rel.max():.3e}"
    assert np.all(r[~nz] == 0)


def test_rmat27_sssp(rmat27):
    g, (rp, col, w), _ = rmat27
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
