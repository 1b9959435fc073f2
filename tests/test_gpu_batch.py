"""Batches of independent graphs (one persistent, graph-captured launch):
every graph's A stream and packed offsets byte-equal to the oracle's own
encoding of that graph (global IDs at bits(n_g - 1), offsets at bits(arcs_g)),
BFS depths from its vertex 0 equal to the oracle's, PageRank after 10
iterations within 1e-4 relative of the FP64 oracle.

Covered: the autotuned schedule, every lanes-per-vertex choice with multi-CTA
teams forced by a small tile, replays, degenerate graphs (one vertex, no arcs,
a path, an isolated vertex 0), invalid input, the device batch generator
against the host one, the team-barrier time limit (a queue member left out on
the host, so the barrier can end only by its limit), and the full 4,096-graph
workload (scales 8..16, edge factors 4..32).
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
ITERS = 10
INF = np.iinfo(np.uint32).max


def host_batch_arrays(b):
    """(vptr, row_ptr, col) numpy views of a gen.Batch or gen.DeviceBatch."""
    if isinstance(b, gen.DeviceBatch):
        return (b.vptr.cpu().numpy().view(np.uint64), b.row_ptr.cpu().numpy().view(np.uint64),
                b.col.cpu().numpy().view(np.uint32))
    return b.vptr, b.row_ptr, b.col


def concat(graphs):
    """gen.Batch from a list of gen.Graph (host)."""
    ns = np.array([g.n for g in graphs], dtype=np.uint64)
    arcs = np.array([g.arcs for g in graphs], dtype=np.uint64)
    vptr = np.zeros(len(graphs) + 1, dtype=np.uint64)
    np.cumsum(ns, out=vptr[1:])
    abase = np.zeros(len(graphs) + 1, dtype=np.uint64)
    np.cumsum(arcs, out=abase[1:])
    rp = np.empty(int(vptr[-1]) + 1, dtype=np.uint64)
    col = np.empty(int(abase[-1]), dtype=np.uint32)
    for i, g in enumerate(graphs):
        rp[int(vptr[i]):int(vptr[i + 1])] = g.row_ptr[:-1] + abase[i]
        col[int(abase[i]):int(abase[i + 1])] = g.col
    rp[-1] = abase[-1]
    z = np.zeros(len(graphs), dtype=np.int64)
    return gen.Batch(vptr=vptr, row_ptr=rp, col=col, scales=z, edge_factors=z)


def to_dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x).view(dt)).cuda()


def create(hb, **kw):
    vptr, rp, col = hb
    return lg.lg_batch_create(to_dev(vptr, np.int64), to_dev(rp, np.int64), to_dev(col, np.int32), **kw)


def check_graph(g, hb, arr, depths, ranks, iters=ITERS):
    """Graph g of the batch against the oracle; returns nothing, asserts."""
    vptr, rp_all, col_all = hb
    v0, v1 = int(vptr[g]), int(vptr[g + 1])
    n = v1 - v0
    a0, a1 = int(rp_all[v0]), int(rp_all[v1])
    rp = (rp_all[v0:v1 + 1] - np.uint64(a0)).astype(np.uint64)
    col = col_all[a0:a1]
    G = arr["graphs"][g]
    assert int(G["n"]) == n and int(G["arcs"]) == a1 - a0
    if n == 0:
        return
    e = oracle.encode(n, rp, col, id_mode=oracle.ID_GLOBAL, off_mode=oracle.OFF_PACKED)
    s, w_o = int(G["s"]), int(G["w_O"])
    assert s == e.s and w_o == e.w_O, f"graph {g}: widths"
    wa = (int(G["arcs"]) * s + 63) // 64
    wo = ((n + 1) * w_o + 63) // 64
    aw, ow = int(G["a_word"]), int(G["o_word"])
    assert np.array_equal(arr["A"][aw:aw + wa], e.A[:wa]), f"graph {g}: A stream"
    assert np.array_equal(arr["O"][ow:ow + wo], e.O[:wo]), f"graph {g}: offsets"
    e.close()
    assert np.array_equal(depths[v0:v1], oracle.bfs(n, rp, col, 0)), f"graph {g}: BFS from vertex 0"
    if iters:
        want = oracle.pagerank(n, rp, col, 0.85, iters)
        got = ranks[v0:v1].astype(np.float64)
        rel = np.abs(got - want) / want
        assert rel.max() <= PR_RTOL, f"graph {g}: PageRank max rel err {rel.max():.3e}"


def run_and_check(b, hb, graphs=None, iters=ITERS, threads=16):
    d, r = lg.lg_batch_run(b, 0.85, iters)
    lg.lg_batch_status(b)
    arr = lg.lg_batch_arrays(b)
    depths = d.cpu().numpy().view(np.uint32)
    ranks = r.cpu().numpy()
    count = arr["graphs"].shape[0]
    todo = range(count) if graphs is None else graphs
    with ThreadPoolExecutor(threads) as ex:  # the oracle calls release the GIL
        list(ex.map(lambda g: check_graph(g, hb, arr, depths, ranks, iters), todo))
    return depths, ranks, arr


@pytest.fixture(scope="module")
def small():
    lg.load(auto_build=True)
    b = gen.rmat_batch(count=256, seed=3, scale_lo=8, scale_hi=13)
    return host_batch_arrays(b)


def test_batch_autotuned(small):
    b = create(small, autotune=True)
    info = b.info()
    assert info["count"] == 256 and info["V"] == int(small[0][-1])
    assert sum(info["graphs_by_lanes"].values()) == 256
    run_and_check(b, small)
    assert info["launches"] >= 1
    b.free()


@pytest.mark.parametrize("lanes", [1, 4, 8, 32])
def test_batch_lanes_with_teams(small, lanes):
    b = create(small, autotune=False, lanes=lanes, tile_arcs=1 << 14)
    info = b.info()
    assert info["teams"] > 0 and info["max_team"] > 8, info
    assert info["graphs_by_lanes"][lanes] == 256
    run_and_check(b, small)
    b.free()


def test_batch_replay_identical(small):
    b = create(small, autotune=False, lanes=8, tile_arcs=1 << 15)
    l0 = lg.lg_kernel_launches()
    d1, r1 = lg.lg_batch_run(b, 0.85, ITERS)
    d1, r1 = d1.clone(), r1.clone()
    d2, r2 = lg.lg_batch_run(b, 0.85, ITERS)
    lg.lg_batch_status(b)
    assert lg.lg_kernel_launches() - l0 == 2  # one graph launch per run
    assert torch.equal(d1, d2) and torch.equal(r1, r2)
    b.free()


def test_batch_iters_zero_and_one(small):
    b = create(small, autotune=False, lanes=4)
    r = torch.full((int(small[0][-1]),), -1.0, device="cuda")
    d, _ = lg.lg_batch_run(b, 0.85, 0, ranks=r)
    lg.lg_batch_status(b)
    assert torch.all(r == -1.0)  # iters = 0 leaves ranks untouched
    run_and_check(b, small, graphs=range(0, 256, 7), iters=1)
    b.free()


def test_batch_degenerate_graphs():
    lg.load(auto_build=True)
    graphs = [
        gen.from_edges(1, np.zeros((0, 2))),                        # one vertex, no arcs
        gen.from_edges(5, np.zeros((0, 2))),                        # five isolated vertices
        gen.from_edges(6, [(i, i + 1) for i in range(5)]),          # path: depth i
        gen.from_edges(4, [(1, 2), (2, 3)]),                        # vertex 0 isolated
        gen.from_edges(2, [(0, 1)]),
        gen.rmat(9, 8, seed=77),
        gen.from_edges(300, [(0, k) for k in range(1, 300)]),       # star, hub 0
    ]
    hb = host_batch_arrays(concat(graphs))
    for lanes in (1, 32):
        b = create(hb, autotune=False, lanes=lanes, tile_arcs=64)
        depths, ranks, _ = run_and_check(b, hb)
        v = hb[0]
        assert list(depths[int(v[2]):int(v[3])]) == [0, 1, 2, 3, 4, 5]
        assert depths[int(v[3])] == 0 and np.all(depths[int(v[3]) + 1:int(v[4])] == INF)
        b.free()


def test_batch_invalid_input():
    lg.load(auto_build=True)
    g = gen.rmat(8, 4, seed=1)
    hb = host_batch_arrays(concat([g, g]))
    vptr, rp, col = hb
    bad = col.copy()
    bad[5] = g.n  # local ID out of range
    with pytest.raises(lg.LgError) as ei:
        create((vptr, rp, bad), autotune=False)
    assert ei.value.status == 1
    bad = col.copy()
    r0 = int(np.argmax(np.diff(g.row_ptr) >= 2))
    j = int(g.row_ptr[r0])
    bad[j], bad[j + 1] = bad[j + 1], bad[j]  # unsorted row
    with pytest.raises(lg.LgError) as ei:
        create((vptr, rp, bad), autotune=False)
    assert ei.value.status == 1
    short = vptr.copy()
    short[-1] -= 1  # graphs do not cover V
    with pytest.raises(lg.LgError) as ei:
        create((short, rp, col), autotune=False)
    assert ei.value.status == 1
    with pytest.raises(lg.LgError):
        create(hb, autotune=False, lanes=3)


def test_batch_team_barrier_time_limit(small):
    """A member of the first team is left out of the queue (on the host): its
    teammates' first barrier can end only by the 20 ms limit.  The run must
    end, report LG_ETIMEOUT, leave every other graph correct, and leave the
    context usable."""
    b = create(small, autotune=False, lanes=8, tile_arcs=1 << 14, wait_limit_us=20000,
               flags=lg.LG_BATCH_FLAG_DROP_MEMBER)
    d, r = lg.lg_batch_run(b, 0.85, ITERS)
    with pytest.raises(lg.LgError) as ei:
        lg.lg_batch_status(b)
    assert ei.value.status == 5  # LG_ETIMEOUT
    arr = lg.lg_batch_arrays(b)
    teams = np.nonzero(arr["graphs"]["team"] > 1)[0]
    work = (arr["graphs"]["arcs"].astype(np.int64) * 2 + arr["graphs"]["n"]) // arr["graphs"]["team"]
    first_team = int(teams[np.argmax(work[teams])])
    others = [g for g in range(256) if g != first_team][::5]
    depths = d.cpu().numpy().view(np.uint32)
    ranks = r.cpu().numpy()
    for g in others:
        check_graph(g, small, arr, depths, ranks)
    b.free()
    ok = create(small, autotune=False, lanes=8, tile_arcs=1 << 14)  # the context still works
    run_and_check(ok, small, graphs=[first_team])
    ok.free()


def test_device_batch_generator_matches_host():
    lg.load(auto_build=True)
    h = gen.rmat_batch(count=48, seed=9, scale_lo=8, scale_hi=12)
    d = gen.rmat_batch_gpu(count=48, seed=9, scale_lo=8, scale_hi=12)
    vptr, rp, col = host_batch_arrays(d)
    assert np.array_equal(vptr, h.vptr) and np.array_equal(rp, h.row_ptr) and np.array_equal(col, h.col)


@pytest.fixture(scope="module")
def full():
    """The full workload: 4,096 R-MAT graphs, scales 8..16, edge factors 4..32."""
    lg.load(auto_build=True)
    d = gen.rmat_batch_gpu(count=4096, seed=3)
    hb = host_batch_arrays(d)
    b = lg.lg_batch_create(d.vptr, d.row_ptr, d.col, autotune=True)
    yield b, hb
    b.free()


def test_batch_full_4096(full):
    b, hb = full
    info = b.info()
    assert info["count"] == 4096 and info["arcs"] == hb[2].shape[0] and info["arcs"] > 1_500_000_000
    run_and_check(b, hb)
