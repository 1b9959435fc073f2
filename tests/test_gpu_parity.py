"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bit-exact: packed A streams, offsets (packed and Elias-Fano, with samples),
permutations, decoded neighborhoods and BFS depths.  PageRank (FP32 on the GPU,
FP64 in the oracle): max relative error per vertex <= 1e-4 after the fixed
iteration count.
"""
import itertools

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg
from helpers import all_graphs, csr_from_edges

pytestmark = pytest.mark.gpu

PR_RTOL = 1e-4
MODES = [(lg.LG_ID_GLOBAL, oracle.ID_GLOBAL), (lg.LG_ID_LOCAL, oracle.ID_LOCAL),
         (lg.LG_ID_LOCAL_GAP, oracle.ID_LOCAL_GAP)]
OFFS = [(lg.LG_OFF_PACKED, oracle.OFF_PACKED), (lg.LG_OFF_EF, oracle.OFF_EF)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lg.load(auto_build=True)
    torch.cuda.init()


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


def encode_both(n, rp, col, w=None, mode=0, off=0, relabel=False, sample=512, weight_bits=0):
    g = lg.lg_encode(dev(rp, np.int64), dev(col, np.int32) if len(col) else torch.empty(0, dtype=torch.int32,
                                                                                         device="cuda"),
                     None if w is None else dev(w, np.int32), id_mode=MODES[mode][0], off_mode=OFFS[off][0],
                     relabel=relabel, select_sample=sample, weight_bits=weight_bits)
    e = oracle.encode(n, rp, col, w, id_mode=MODES[mode][1], off_mode=OFFS[off][1], relabel=relabel,
                      sample=sample, weight_bits=weight_bits)
    return g, e


def assert_arrays_equal(g, e):
    a = lg.lg_arrays_get(g)
    st = lg.lg_stats_get(g)
    assert st["bits_A"] == e.bits_A and st["s"] == e.s
    assert np.array_equal(a["A"], e.A), "A stream"
    if e.off_mode == oracle.OFF_PACKED:
        assert st["w_O"] == e.w_O
        assert np.array_equal(a["O"], e.O), "packed offsets"
    else:
        assert st["ef_l"] == e.ef_l
        assert np.array_equal(a["ef_low"], e.ef_low), "EF low bits"
        assert np.array_equal(a["ef_high"], e.ef_high), "EF high bits"
        assert np.array_equal(a["ef_samples"], e.samples), "EF samples"
    if e.relabel:
        assert np.array_equal(a["perm"], e.perm) and np.array_equal(a["inv_perm"], e.inv_perm)


def assert_neighbors(g, rp, col, n, w=None, vertices=None):
    vs = np.arange(n, dtype=np.uint32) if vertices is None else np.asarray(vertices, dtype=np.uint32)
    if w is None:
        off, ids = lg.lg_neighbors(g, dev(vs, np.int32))
    else:
        off, ids, wts = lg.lg_neighbors(g, dev(vs, np.int32), with_weights=True)
    off = off.cpu().numpy().view(np.uint64)
    ids = ids.cpu().numpy().view(np.uint32)
    deg = (rp[vs.astype(np.int64) + 1] - rp[vs]).astype(np.uint64)
    assert np.array_equal(np.diff(off), deg)
    want = np.concatenate([col[rp[v]:rp[v + 1]] for v in vs]) if len(vs) else np.zeros(0, np.uint32)
    assert np.array_equal(ids, want)
    if w is not None:
        ww = np.concatenate([w[rp[v]:rp[v + 1]] for v in vs]) if len(vs) else np.zeros(0, np.uint32)
        assert np.array_equal(wts.cpu().numpy().view(np.uint32), ww)


def stored_csr(n, rp, col, w=None, perm=None):
    """The CSR in stored order: the input, or with a relabel row perm[v] =
    sorted perm of N_v (weights follow their arcs)."""
    if perm is None:
        return rp, col, w
    perm = np.asarray(perm, dtype=np.int64)
    deg = np.diff(rp).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    r, c = perm[src], perm[np.asarray(col, dtype=np.int64)]
    order = np.lexsort((c, r))
    nrp = np.zeros(n + 1, dtype=np.int64)
    nrp[1:] = np.cumsum(np.bincount(r, minlength=n))
    nw = None if w is None else np.asarray(w)[order]
    return nrp.astype(np.uint64), c[order].astype(np.uint32), nw


def assert_decode(g, n, rp, col, w=None, perm=None):
    want_rp, want_col, want_w = stored_csr(n, rp, col, w, perm)
    if w is None:
        grp, gcol = lg.lg_decode(g)
    else:
        grp, gcol, gw = lg.lg_decode(g, with_weights=True)
        assert np.array_equal(gw.cpu().numpy().view(np.uint32), want_w), "decoded weights"
    assert np.array_equal(grp.cpu().numpy().view(np.uint64), np.asarray(want_rp, dtype=np.uint64)), "decoded row_ptr"
    assert np.array_equal(gcol.cpu().numpy().view(np.uint32), np.asarray(want_col, dtype=np.uint32)), "decoded col"


def assert_bfs(g, n, rp, col, sources):
    d = lg.lg_bfs(g, dev(np.asarray(sources, dtype=np.uint32), np.int32)).cpu().numpy().view(np.uint32)
    for i, s in enumerate(sources):
        want = oracle.bfs(n, rp, col, int(s))
        assert np.array_equal(d[i], want), f"BFS depths from source {s}"


def assert_pagerank(g, n, rp, col, iters=20, personalize=None, damping=0.85):
    r = lg.lg_pagerank(g, damping, iters, personalize=personalize).cpu().numpy().astype(np.float64)
    want = oracle.pagerank(n, rp, col, damping, iters, -1 if personalize is None else personalize)
    nz = want > 0
    rel = np.abs(r[nz] - want[nz]) / want[nz]
    assert rel.max(initial=0.0) <= PR_RTOL, f"PageRank max rel err {rel.max():.3e}"
    assert np.all(np.abs(r[~nz]) <= 1e-30)


# ------------------------------------------------------------------ tiny graphs, exhaustive
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_exhaustive_tiny_graphs_all_modes(n):
    for edges in all_graphs(n):
        rp, col, _ = csr_from_edges(n, edges)
        for mode, off, relabel in itertools.product(range(3), range(2), (False, True)):
            g, e = encode_both(n, rp, col, mode=mode, off=off, relabel=relabel, sample=64)
            assert_arrays_equal(g, e)
            assert_neighbors(g, rp, col, n)
            assert_decode(g, n, rp, col, perm=e.perm if relabel else None)
            g.free()


@pytest.mark.parametrize("seed", range(3))
def test_five_vertex_graphs_sampled(seed):
    rng = np.random.default_rng(seed)
    graphs = list(all_graphs(5))
    for idx in rng.choice(len(graphs), size=40, replace=False):
        rp, col, _ = csr_from_edges(5, graphs[idx])
        for mode, off in itertools.product(range(3), range(2)):
            g, e = encode_both(5, rp, col, mode=mode, off=off, relabel=bool(idx & 1), sample=64)
            assert_arrays_equal(g, e)
            assert_neighbors(g, rp, col, 5)
            assert_bfs(g, 5, rp, col, list(range(5)))
            assert_pagerank(g, 5, rp, col, iters=7)


# ------------------------------------------------------------------ special shapes
SHAPES = {
    "single_vertex": (1, []),
    "no_edges": (37, []),
    "isolated_runs": (700, [(0, 699), (5, 6), (650, 3)]),
    "star": (2000, [(0, i) for i in range(1, 2000)]),
    "path": (1500, [(i, i + 1) for i in range(1499)]),
    "complete": (64, [(i, j) for i in range(64) for j in range(i + 1, 64)]),
    "pow2_n": (1024, [(i, (i * 37 + 11) % 1024) for i in range(1024)]),
    "pow2_plus1_n": (1025, [(i, (i * 37 + 11) % 1025) for i in range(1025)]),
}


@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("mode,off", list(itertools.product(range(3), range(2))))
def test_special_shapes(shape, mode, off):
    n, edges = SHAPES[shape]
    rp, col, _ = csr_from_edges(n, edges)
    for relabel in (False, True):
        g, e = encode_both(n, rp, col, mode=mode, off=off, relabel=relabel, sample=64)
        assert_arrays_equal(g, e)
        assert_neighbors(g, rp, col, n)
        srcs = sorted({0, n - 1, n // 2})
        assert_bfs(g, n, rp, col, srcs)
        assert_pagerank(g, n, rp, col, iters=10)
        g.free()


# ------------------------------------------------------------------ R-MAT scale 16 (the small config)
@pytest.fixture(scope="module")
def rmat16():
    return gen.rmat_s16_ef16()


@pytest.mark.parametrize("mode,off", list(itertools.product(range(3), range(2))))
def test_rmat16_streams_and_decode(rmat16, mode, off):
    g0 = rmat16
    for relabel in (False, True):
        g, e = encode_both(g0.n, g0.row_ptr, g0.col, mode=mode, off=off, relabel=relabel)
        assert_arrays_equal(g, e)
        assert_neighbors(g, g0.row_ptr, g0.col, g0.n)
        g.free()


def test_rmat16_global_packed_widths(rmat16):
    g, e = encode_both(rmat16.n, rmat16.row_ptr, rmat16.col, mode=0, off=0)
    st = lg.lg_stats_get(g)
    assert st["s"] == 16 and st["w_O"] == 21
    assert st["bits_A"] == 16 * rmat16.arcs


@pytest.mark.parametrize("mode,off", [(0, 0), (2, 1), (1, 1), (0, 1)])
def test_rmat16_bfs_64_sources(rmat16, mode, off):
    g0 = rmat16
    src = gen.sources(g0, 64, seed=1)
    g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=mode, off=off, relabel=(mode == 2))
    assert_bfs(g, g0.n, g0.row_ptr, g0.col, src)


@pytest.mark.parametrize("S", [1, 3, 16, 17, 33, 64, 65, 100])
def test_rmat16_bfs_source_counts(rmat16, S):
    g0 = rmat16
    src = gen.sources(g0, S, seed=S)
    g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=2, off=1, relabel=True)
    assert_bfs(g, g0.n, g0.row_ptr, g0.col, src)


@pytest.mark.parametrize("mode,off", list(itertools.product(range(3), range(2))))
def test_rmat16_pagerank_20(rmat16, mode, off):
    g0 = rmat16
    g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=mode, off=off, relabel=(off == 1))
    assert_pagerank(g, g0.n, g0.row_ptr, g0.col, iters=20)


def test_rmat16_personalized_pagerank(rmat16):
    g0 = rmat16
    g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=2, off=1, relabel=True)
    for s in gen.sources(g0, 3, seed=5):
        assert_pagerank(g, g0.n, g0.row_ptr, g0.col, iters=10, personalize=int(s))


def test_csr32_baseline_same_kernels(rmat16):
    g0 = rmat16
    for relabel in (False, True):
        g = lg.lg_encode(dev(g0.row_ptr, np.int64), dev(g0.col, np.int32), id_mode=lg.LG_ID_CSR32, relabel=relabel)
        assert_neighbors(g, g0.row_ptr, g0.col, g0.n)
        assert_bfs(g, g0.n, g0.row_ptr, g0.col, gen.sources(g0, 16, seed=2))
        assert_pagerank(g, g0.n, g0.row_ptr, g0.col, iters=20)


# ------------------------------------------------------------------ weights
@pytest.mark.parametrize("wbits,maxw", [(0, 1), (0, 255), (0, 256), (24, 200), (32, 7)])
def test_weighted_global(wbits, maxw):
    g0 = gen.rmat(11, 8, seed=7, weighted=True)
    w = (g0.weights.astype(np.uint64) * maxw // 255).astype(np.uint32)
    w[w == 0] = 1 if maxw >= 1 else 0
    w[np.argmax(g0.col)] = maxw  # make the maximum appear (both arcs need not agree for decode parity)
    for off in range(2):
        g, e = encode_both(g0.n, g0.row_ptr, g0.col, w, mode=0, off=off, weight_bits=wbits)
        assert_arrays_equal(g, e)
        assert_neighbors(g, g0.row_ptr, g0.col, g0.n, w=w)
        assert_bfs(g, g0.n, g0.row_ptr, g0.col, [0, 5])
    g = lg.lg_encode(dev(g0.row_ptr, np.int64), dev(g0.col, np.int32), dev(w, np.int32), id_mode=lg.LG_ID_CSR32)
    assert_neighbors(g, g0.row_ptr, g0.col, g0.n, w=w)


def test_weighted_relabel_and_35_bit_records():
    g0 = gen.rmat(12, 16, seed=8, weighted=True)
    g, e = encode_both(g0.n, g0.row_ptr, g0.col, g0.weights, mode=0, off=1, relabel=True, weight_bits=23)
    assert lg.lg_stats_get(g)["s"] + 23 == 35
    assert_arrays_equal(g, e)
    assert_neighbors(g, g0.row_ptr, g0.col, g0.n, w=g0.weights)


@pytest.mark.parametrize("relabel", [True, lg.LG_RELABEL_GREEDY])
@pytest.mark.parametrize("weighted", [False, True])
def test_relabel_every_row_size_class(weighted, relabel):
    """Relabeling re-sorts every row: degrees on both sides of each sort size
    class boundary (sub-warp, warp, register networks of 1..8 warps, radix).
    DM order puts the rows above 4,096 keys first (sorted where they lie); the
    greedy order scatters them (gathered, sorted, scattered back)."""
    rng = np.random.default_rng(11)
    degs = [0, 1, 2, 3, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512,
            513, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 6000, 8191, 8192, 8193]
    n = 9000
    deg = np.zeros(n, dtype=np.int64)
    rows = rng.permutation(n)[:5 * len(degs)]
    deg[rows] = np.repeat(degs, 5)
    deg[deg == 0] = rng.integers(0, 40, size=int((deg == 0).sum()))
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(deg)
    col = np.concatenate([np.sort(rng.choice(n, int(d), replace=False)) for d in deg]).astype(np.uint32)
    w = rng.integers(0, 1 << 20, size=len(col)).astype(np.uint32) if weighted else None
    for mode in (0, 2):
        g, e = encode_both(n, rp, col, w, mode=mode, off=1, relabel=relabel,
                           weight_bits=20 if weighted and mode == 0 else 0)
        assert_arrays_equal(g, e)
        assert_neighbors(g, rp, col, n, w=w if weighted and mode == 0 else None)
        if weighted:
            break


@pytest.mark.parametrize("mode,off", list(itertools.product(range(3), range(2))))
@pytest.mark.parametrize("relabel", [False, True])
def test_decode_whole_graph(rmat16, mode, off, relabel):
    """lg_decode over R-MAT 2^16 (hubs on the heavy schedule, light runs per
    warp): the input CSR, or the relabeled CSR in stored order."""
    g0 = rmat16
    g, e = encode_both(g0.n, g0.row_ptr, g0.col, mode=mode, off=off, relabel=relabel)
    assert_decode(g, g0.n, g0.row_ptr, g0.col, perm=e.perm if relabel else None)


@pytest.mark.parametrize("relabel", [False, True])
def test_decode_csr32_and_weights(rmat16, relabel):
    g0 = rmat16
    g = lg.lg_encode(dev(g0.row_ptr, np.int64), dev(g0.col, np.int32), id_mode=lg.LG_ID_CSR32, relabel=relabel)
    perm = lg.lg_arrays_get(g)["perm"] if relabel else None
    assert_decode(g, g0.n, g0.row_ptr, g0.col, perm=perm)
    w0 = gen.rmat(12, 16, seed=8, weighted=True)
    g, e = encode_both(w0.n, w0.row_ptr, w0.col, w0.weights, mode=0, off=1, relabel=relabel, weight_bits=23)
    assert_decode(g, w0.n, w0.row_ptr, w0.col, w=w0.weights, perm=e.perm if relabel else None)


def test_decode_errors(rmat16):
    g0 = rmat16
    g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=2, off=1)
    lib = lg.load()
    rp = torch.empty(g0.n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(len(g0.col), dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.lg_decode(g.handle, rp.data_ptr(), col.data_ptr(), None, len(g0.col) - 1, st) == 4  # LG_ERANGE
    assert lib.lg_decode(g.handle, rp.data_ptr(), col.data_ptr(), col.data_ptr(), len(g0.col), st) == 1  # no weights
    assert lib.lg_decode(None, rp.data_ptr(), col.data_ptr(), None, len(g0.col), st) == 1


# ------------------------------------------------------------------ queries and errors
def test_neighbors_random_queries_with_repeats(rmat16):
    g0 = rmat16
    rng = np.random.default_rng(3)
    q = rng.integers(0, g0.n, size=1000).astype(np.uint32)
    q[:10] = q[0]
    for mode, off in itertools.product(range(3), range(2)):
        g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=mode, off=off, relabel=(mode > 0))
        assert_neighbors(g, g0.row_ptr, g0.col, g0.n, vertices=q)


def test_neighbors_capacity_and_range_errors(rmat16):
    g0 = rmat16
    g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=2, off=1)
    lib = lg.load()
    vs = dev(np.array([1, 2, 3], dtype=np.uint32), np.int32)
    off = torch.empty(4, dtype=torch.int64, device="cuda")
    ids = torch.empty(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.lg_neighbors(g.handle, vs.data_ptr(), 3, off.data_ptr(), ids.data_ptr(), None, 0, st)
    assert rc == 4  # LG_ERANGE, offsets written
    deg = g0.row_ptr[[2, 3, 4]] - g0.row_ptr[[1, 2, 3]]
    assert np.array_equal(np.diff(off.cpu().numpy()), deg.astype(np.int64))
    bad = dev(np.array([g0.n], dtype=np.uint32), np.int32)
    with pytest.raises(lg.LgError) as ei:
        lg.lg_neighbors(g, bad)
    assert ei.value.status == 1
    with pytest.raises(lg.LgError):
        lg.lg_bfs(g, bad)
    with pytest.raises(lg.LgError):
        lg.lg_pagerank(g, 0.85, 3, personalize=g0.n)


def test_invalid_csr_is_rejected_without_fault():
    rp, col, _ = csr_from_edges(6, [(0, 1), (1, 2), (2, 3)])
    bad_cases = []
    c = col.copy(); c[0] = 99; bad_cases.append((rp, c))              # id out of range
    c = col.copy(); c[1], c[2] = c[2], c[1]; bad_cases.append((rp, c))  # row out of order
    r = rp.copy(); r[2] = r[1] - 1 if r[1] else 0; bad_cases.append((r, col))  # row_ptr decreasing
    r = rp.copy(); r[-1] = 10**9; bad_cases.append((r, col))          # row_ptr past the end
    for r, c in bad_cases:
        with pytest.raises(lg.LgError) as ei:
            lg.lg_encode(dev(r, np.int64), dev(c, np.int32), id_mode=lg.LG_ID_LOCAL_GAP, off_mode=lg.LG_OFF_EF)
        assert ei.value.status == 1
    # asymmetric input is caught when asked
    rp2 = np.array([0, 1, 1], dtype=np.uint64)
    col2 = np.array([1], dtype=np.uint32)
    with pytest.raises(lg.LgError):
        lg.lg_encode(dev(rp2, np.int64), dev(col2, np.int32), check_symmetric=True)
    # the device is still usable afterwards
    g = lg.lg_encode(dev(rp, np.int64), dev(col, np.int32))
    assert_neighbors(g, rp, col, 6)


def test_unsupported_and_bad_options():
    rp, col, _ = csr_from_edges(4, [(0, 1)])
    w = np.array([3, 3], dtype=np.uint32)
    with pytest.raises(lg.LgError) as ei:
        lg.lg_encode(dev(rp, np.int64), dev(col, np.int32), dev(w, np.int32), id_mode=lg.LG_ID_LOCAL)
    assert ei.value.status == 6
    with pytest.raises(lg.LgError):
        lg.lg_encode(dev(rp, np.int64), dev(col, np.int32), off_mode=lg.LG_OFF_EF, select_sample=100)
    with pytest.raises(lg.LgError):
        lg.lg_encode(dev(rp, np.int64), dev(col, np.int32), dev(w, np.int32), weight_bits=1)


def test_pagerank_zero_iterations_and_sum_rule(rmat16):
    g0 = rmat16
    g, _ = encode_both(g0.n, g0.row_ptr, g0.col, mode=2, off=1, relabel=True)
    r0 = lg.lg_pagerank(g, 0.85, 0).cpu().numpy()
    assert np.allclose(r0, 1.0 / g0.n)
    r = lg.lg_pagerank(g, 0.85, 20).cpu().numpy().astype(np.float64)
    iso = g0.degrees() == 0
    assert abs(r.sum() - (1.0 - iso.sum() * 0.85 / g0.n)) < 1e-3


# ------------------------------------------------------------------ heavy-vertex schedule
@pytest.fixture
def small_schedule(monkeypatch):
    """Force most vertices onto the warp schedule and split them into many items."""
    monkeypatch.setenv("LG_HEAVY_MIN", "6")
    monkeypatch.setenv("LG_HEAVY_SEG", "40")


@pytest.mark.parametrize("mode,off", list(itertools.product(range(3), range(2))))
def test_heavy_schedule_paths(rmat16, small_schedule, mode, off):
    g0 = rmat16
    g, e = encode_both(g0.n, g0.row_ptr, g0.col, mode=mode, off=off, relabel=(mode == 2))
    st = lg.lg_stats_get(g)
    assert st["bytes_schedule"] > 0
    assert_arrays_equal(g, e)  # the schedule is derived data, the format is unchanged
    assert_bfs(g, g0.n, g0.row_ptr, g0.col, gen.sources(g0, 20, seed=4))
    assert_pagerank(g, g0.n, g0.row_ptr, g0.col, iters=20)


def test_heavy_schedule_csr32(rmat16, small_schedule):
    g0 = rmat16
    g = lg.lg_encode(dev(g0.row_ptr, np.int64), dev(g0.col, np.int32), id_mode=lg.LG_ID_CSR32)
    assert_bfs(g, g0.n, g0.row_ptr, g0.col, gen.sources(g0, 5, seed=6))
    assert_pagerank(g, g0.n, g0.row_ptr, g0.col, iters=20)


@pytest.mark.parametrize("mode,off", list(itertools.product(range(3), range(2))))
def test_split_hubs_default_schedule(mode, off):
    # two hubs of degree 9000 and 5000 (3 and 2 items at 4096 fields), leaves
    # shared between them, and a tail path
    n = 12000
    edges = [(0, i) for i in range(1, 9001)] + [(1, i) for i in range(4000, 9000)]
    edges += [(i, i + 1) for i in range(9001, n - 1)]
    rp, col, _ = csr_from_edges(n, edges)
    for relabel in (False, True):
        g, e = encode_both(n, rp, col, mode=mode, off=off, relabel=relabel)
        assert_arrays_equal(g, e)
        assert_neighbors(g, rp, col, n, vertices=[0, 1, 2, 4500, 9001, n - 1])
        assert_bfs(g, n, rp, col, [0, 4500, n - 1])
        assert_pagerank(g, n, rp, col, iters=15)
