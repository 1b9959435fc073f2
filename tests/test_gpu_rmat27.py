"""Full-size parity on the largest configuration: R-MAT scale 27 (134,217,728
vertices, edge factor 16, ~4.22e9 stored arcs), integer weights in [1, 255]
stored at 8 bits, global 27-bit IDs, Elias-Fano offsets -- 35-bit records and
bit positions far past 2^32.  The graph is built on the device by the seeded
generator (the same edges as the host generator) and copied to the host for
the oracle.  It is encoded twice: in the generator's order and, as the
benchmark runs it, in DM order (Section 5.6: degree descending, ties by ID).

Generator order, compared with the oracle in full: the whole Elias-Fano offset
structure, the whole A stream (1.48e11 bits, window by window with the
oracle's bit-by-bit encoder on every host core), the whole-graph decode (the
input CSR itself).

DM order: the permutation in full against its definition; the Elias-Fano
arrays in full; 2,600 windows of the A stream (the hub rows first) against the
oracle's encoder over the relabeled rows; the whole-graph decode in full
(row offsets equal, every row strictly increasing, every row the relabeled
neighborhood with its weights: per-row sums of a 64-bit hash); all 16 BFS depth rows and
every 20-iteration PageRank value (1e-4 relative) against the oracle on the
input CSR; SSSP over the 8-bit weights from one source (Dijkstra; three more
sources by the defining properties); 4,000 sampled neighborhoods with weights.
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


@pytest.fixture(scope="module")
def rmat27_dm(rmat27):
    """The same graph in DM order (the benchmark's encoding), with the
    relabeled CSR's definition computed here: label of v = rank of v in
    (degree descending, ID ascending)."""
    _, (rp, col, w), (rp_d, col_d, w_d) = rmat27
    g = lg.lg_encode(rp_d, col_d, w_d, id_mode=lg.LG_ID_GLOBAL, off_mode=lg.LG_OFF_EF, weight_bits=8, relabel=True)
    n = rp.shape[0] - 1
    deg = np.diff(rp).astype(np.int64)
    inv = np.lexsort((np.arange(n), -deg)).astype(np.uint32)  # stored -> original
    perm = np.empty(n, dtype=np.uint32)
    perm[inv] = np.arange(n, dtype=np.uint32)
    srp = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(deg[inv], out=srp[1:])
    yield g, perm, inv, srp
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


def test_rmat27_dm_permutation_and_offsets(rmat27, rmat27_dm):
    """perm / inv_perm equal the DM definition; the relabeled graph's
    Elias-Fano arrays equal the oracle's over the relabeled row offsets."""
    g, perm, inv, srp = rmat27_dm
    a = lg.lg_arrays_device(g)
    assert np.array_equal(a["perm"].cpu().numpy().view(np.uint32), perm)
    assert np.array_equal(a["inv_perm"].cpu().numpy().view(np.uint32), inv)
    low, high, smp, l = oracle.ef_build(srp, sample=512)
    assert lg.lg_stats_get(g)["ef_l"] == l
    assert np.array_equal(a["ef_low"].cpu().numpy().view(np.uint64), low)
    assert np.array_equal(a["ef_high"].cpu().numpy().view(np.uint64), high)
    assert np.array_equal(a["ef_samples"].cpu().numpy().view(np.uint64), smp)


def test_rmat27_dm_A_windows(rmat27, rmat27_dm):
    """2,600 windows of 70 words (128 records, starting on a word) of the DM
    graph's A stream equal the oracle's encoder over the relabeled rows: the
    first 500 windows (the hubs' rows), 2,000 at random, the last 100."""
    _, (rp, col, w), _ = rmat27
    g, perm, inv, srp = rmat27_dm
    A = lg.lg_arrays_device(g)["A"]
    arcs = col.shape[0]
    nwin = arcs // 128
    rng = np.random.default_rng(35)
    wins = np.unique(np.concatenate([np.arange(500), rng.integers(0, nwin, 2000), np.arange(nwin - 100, nwin)]))
    cache = {}

    def sorted_slice(i, r0, r1):
        """Ranks [r0, r1) of relabeled row i (sorted new labels, their
        weights): a full sort for short rows and the first windows' rows, a
        selection by two order statistics for a random window in a long row."""
        v = int(inv[i])
        lo, hi = int(rp[v]), int(rp[v + 1])
        if i in cache or hi - lo <= 8192 or len(cache) < 8:
            if i not in cache:
                keys = perm[col[lo:hi]]
                o = np.argsort(keys, kind="stable")
                cache[i] = (keys[o], w[lo:hi][o])
            k, ww = cache[i]
            return k[r0:r1], ww[r0:r1]
        keys = perm[col[lo:hi]]
        part = np.partition(keys, [r0, r1 - 1])
        m = (keys >= part[r0]) & (keys <= part[r1 - 1])  # labels in a row are distinct
        k, ww = keys[m], w[lo:hi][m]
        o = np.argsort(k, kind="stable")
        return k[o], ww[o]

    for k in wins:
        j0, j1 = int(k) * 128, int(k) * 128 + 128
        # (numpy compares a uint64 array with a Python int by converting the whole array)
        i0 = int(np.searchsorted(srp, np.uint64(j0), side="right")) - 1
        i1 = int(np.searchsorted(srp, np.uint64(j1 - 1), side="right")) - 1
        parts = [sorted_slice(i, max(j0, int(srp[i])) - int(srp[i]), min(j1, int(srp[i + 1])) - int(srp[i]))
                 for i in range(i0, i1 + 1)]
        c = np.ascontiguousarray(np.concatenate([p[0] for p in parts]))
        ww = np.ascontiguousarray(np.concatenate([p[1] for p in parts]))
        want = oracle.global_words(c, ww, 27, 8, 0, 70)
        w0 = j0 * 35 // 64
        got = A[w0:w0 + 70].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), f"DM A window at record {j0}"
        if len(cache) > 4096:
            cache.clear()


def _hash(x):
    x = x.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    return x ^ (x >> np.uint64(29))


def test_rmat27_dm_whole_decode(rmat27, rmat27_dm):
    """lg_decode of the DM graph in full: row offsets equal the relabeled
    ones, every row is strictly increasing, and every row holds the relabeled
    neighborhood with its weights (equal per-row sums of a 64-bit hash of
    (original neighbor, weight)); whole rows are compared ~2^28 arcs at a time."""
    _, (rp, col, w), _ = rmat27
    g, perm, inv, srp = rmat27_dm
    drp, dcol, dw = lg.lg_decode(g, with_weights=True)
    assert np.array_equal(drp.cpu().numpy().view(np.uint64), srp)
    del drp
    n = rp.shape[0] - 1
    CA = 1 << 28  # arcs per chunk of whole rows
    r0 = 0
    while r0 < n:
        r1 = int(np.searchsorted(srp, srp[r0] + np.uint64(CA), side="right")) - 1
        r1 = min(n, max(r1, r0 + 1))
        a0, a1 = int(srp[r0]), int(srp[r1])
        if a0 < a1:
            sc = dcol[a0:a1].cpu().numpy().view(np.uint32)
            sw = dw[a0:a1].cpu().numpy().view(np.uint32)
            d = np.diff(srp[r0:r1 + 1]).astype(np.int64)
            nz = d > 0
            starts = (srp[r0:r1][nz] - np.uint64(a0)).astype(np.int64)
            inc = np.ones(a1 - a0, dtype=bool)
            inc[1:] = sc[1:] > sc[:-1]
            inc[starts] = True  # a row start is not compared with the row before
            assert inc.all(), f"decoded rows not strictly increasing in rows [{r0}, {r1})"
            got = np.add.reduceat(_hash(inv[sc].astype(np.uint64) * np.uint64(256) + sw), starts)
            v = inv[r0:r1][nz].astype(np.int64)
            lo, dd = rp[v].astype(np.int64), d[nz]
            cstart = np.concatenate([[0], np.cumsum(dd)[:-1]])
            idx = np.repeat(lo - cstart, dd) + np.arange(int(dd.sum()), dtype=np.int64)
            want = np.add.reduceat(_hash(col[idx].astype(np.uint64) * np.uint64(256) + w[idx]), cstart)
            assert np.array_equal(got, want), f"decoded rows differ from the relabeled neighborhoods in [{r0}, {r1})"
        r0 = r1
    del dcol, dw
    torch.cuda.empty_cache()


def test_rmat27_sampled_neighborhoods(rmat27, rmat27_dm):
    _, (rp, col, w), _ = rmat27
    g = rmat27_dm[0]
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


def test_rmat27_bfs_16_sources(rmat27, rmat27_dm):
    """DM graph: all 16 depth rows equal the oracle's FIFO BFS on the input CSR."""
    _, (rp, col, _), _ = rmat27
    g = rmat27_dm[0]
    n = rp.shape[0] - 1
    src = _sources(n, rp)
    d = lg.lg_bfs(g, torch.from_numpy(src.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    with ThreadPoolExecutor(min(16, NPROC)) as ex:  # the oracle runs one BFS per thread
        want = ex.map(lambda s: oracle.bfs(n, rp, col, int(s)), src)
        for i, wd in enumerate(want):
            assert np.array_equal(d[i], wd), f"source {src[i]}"


def test_rmat27_pagerank_20(rmat27, rmat27_dm):
    """DM graph: every vertex within 1e-4 relative of the FP64 oracle after
    the 20 iterations the workload runs."""
    _, (rp, col, _), _ = rmat27
    g = rmat27_dm[0]
    n = rp.shape[0] - 1
    r = lg.lg_pagerank(g, 0.85, 20).cpu().numpy().astype(np.float64)
    want = oracle.pagerank(n, rp, col, 0.85, 20, threads=NPROC)
    nz = want > 0
    rel = np.abs(r[nz] - want[nz]) / want[nz]
    assert rel.max() <= 1e-4, f"max rel err {rel.max():.3e}"
    assert np.all(r[~nz] == 0)


def test_rmat27_sssp(rmat27, rmat27_dm):
    """DM graph (the SSSP benchmark's encoding): distances from one source
    equal Dijkstra on the input CSR; three more sources by the defining
    properties."""
    _, (rp, col, w), _ = rmat27
    g = rmat27_dm[0]
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
