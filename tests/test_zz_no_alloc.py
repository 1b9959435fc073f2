"""lg_pagerank_noalloc: the PageRank entry point for callers that cannot
allocate device memory (their memory belongs to another allocator or a fixed
budget, or their loop cannot take cudaFree's implicit synchronization).

It is called here through the C ABI (and once through the Python wrapper) and
must give the results of lg_pagerank and of the FP64 oracle (1e-4 relative
per vertex), on two calls in a row (the second reuses the library's scratch
array as the first left it), without allocating: the library's device pool
and torch's allocator hold the same bytes before and after.  One graph has a
hub whose degree exceeds the split size of the heavy-vertex schedule, so the
scratch region of the split vertices' partial sums is exercised.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg

pytestmark = pytest.mark.gpu

RTOL = 1e-4  # the PageRank tolerance of the parity tests
SPLIT = 4096  # fields per heavy-schedule item (the library default)


def _cuda(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


def _call(lib, g, damping, iters, out, personalize=None):
    ps = None if personalize is None else ctypes.byref(ctypes.c_uint32(personalize))
    return lib.lg_pagerank_noalloc(g.handle, ctypes.c_float(damping), iters, ps, out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)


def _hub_graph():
    """R-MAT scale 14 plus one hub adjacent to 3 * SPLIT + 17 vertices."""
    base = gen.rmat(14, 8, seed=21)
    rp, col = base.row_ptr, base.col
    src = np.repeat(np.arange(base.n, dtype=np.uint32), np.diff(rp).astype(np.int64))
    edges = np.stack([src, col], axis=1)
    edges = edges[edges[:, 0] < edges[:, 1]]
    hub = np.stack([np.zeros(3 * SPLIT + 17, dtype=np.uint32),
                    np.arange(1, 3 * SPLIT + 18, dtype=np.uint32)], axis=1)
    return gen.from_edges(base.n, np.concatenate([edges, hub]))


def _graphs():
    return {"rmat16": gen.rmat_s16_ef16(), "hub": _hub_graph()}


@pytest.fixture(scope="module")
def inputs():
    return _graphs()


def _usage():
    torch.cuda.synchronize()
    return lg.lg_pool_usage(torch.cuda.current_device()), torch.cuda.memory_allocated()


@pytest.mark.parametrize("name,mode,off,relabel", [("rmat16", lg.LG_ID_LOCAL_GAP, lg.LG_OFF_EF, True),
                                                   ("rmat16", lg.LG_ID_GLOBAL, lg.LG_OFF_PACKED, False),
                                                   ("hub", lg.LG_ID_GLOBAL, lg.LG_OFF_EF, False),
                                                   ("hub", lg.LG_ID_LOCAL_GAP, lg.LG_OFF_EF, True)])
def test_noalloc_matches_pagerank_and_oracle_twice(inputs, name, mode, off, relabel):
    lib = lg.load(auto_build=True)
    g0 = inputs[name]
    g = lg.lg_encode(_cuda(g0.row_ptr, np.int64), _cuda(g0.col, np.int32), id_mode=mode, off_mode=off,
                     relabel=relabel)
    if name == "hub":
        assert lg.lg_stats_get(g)["max_degree"] > 2 * SPLIT  # the hub is split into several items
    outs = [torch.full((g0.n,), -1.0, dtype=torch.float32, device="cuda") for _ in range(2)]
    for personalize in (None, int(gen.sources(g0, 1, seed=3)[0])):
        want = lg.lg_pagerank(g, 0.85, 20, personalize=personalize).cpu().numpy()
        ref = oracle.pagerank(g0.n, g0.row_ptr, g0.col, 0.85, 20, personalize=-1 if personalize is None
                              else personalize)
        before = _usage()
        for out in outs:  # two calls in a row
            assert _call(lib, g, 0.85, 20, out, personalize) == 0, lg.lg_last_error()
        after = _usage()
        assert after == before, f"device memory changed: {before} -> {after}"
        for out in outs:
            got = out.cpu().numpy()
            nz = want > 0
            assert np.all(np.abs(got[nz] - want[nz]) <= RTOL * want[nz])
            assert np.all(got[~nz] == want[~nz])
            rz = ref > 0
            rel = np.abs(got[rz].astype(np.float64) - ref[rz]) / ref[rz]
            assert rel.max() <= RTOL, f"max rel err vs oracle {rel.max():.3e}"
            assert np.all(got[~rz] == 0)


def test_noalloc_python_wrapper_and_zero_iterations(inputs):
    lg.load(auto_build=True)
    g0 = inputs["rmat16"]
    g = lg.lg_encode(_cuda(g0.row_ptr, np.int64), _cuda(g0.col, np.int32), id_mode=lg.LG_ID_LOCAL_GAP,
                     off_mode=lg.LG_OFF_EF, relabel=True)
    out = torch.empty(g0.n, dtype=torch.float32, device="cuda")
    got = lg.lg_pagerank_noalloc(g, 0.85, 5, out).cpu().numpy().astype(np.float64)
    ref = oracle.pagerank(g0.n, g0.row_ptr, g0.col, 0.85, 5)
    assert (np.abs(got - ref) / ref).max() <= RTOL
    # zero iterations: r_0, exactly as lg_pagerank writes it
    for personalize in (None, 7):
        a = lg.lg_pagerank_noalloc(g, 0.85, 0, out, personalize=personalize).cpu().numpy()
        b = lg.lg_pagerank(g, 0.85, 0, personalize=personalize).cpu().numpy()
        assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        lg.lg_pagerank_noalloc(g, 0.85, 5, out[:-1])
    with pytest.raises(TypeError):
        lg.lg_pagerank_noalloc(g, 0.85, 5, out.double())


def test_noalloc_rejects_graphs_beyond_its_limit():
    lib = lg.load(auto_build=True)
    n = (1 << 20) + 1
    rp = np.ones(n + 1, dtype=np.uint64)  # one edge 0 - (n-1)
    rp[0] = 0
    rp[-1] = 2
    col = np.array([n - 1, 0], dtype=np.uint32)
    g = lg.lg_encode(_cuda(rp, np.int64), _cuda(col, np.int32))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    assert _call(lib, g, 0.85, 5, out) == 4  # LG_ERANGE
    assert "at most 1048576 vertices" in lg.lg_last_error()
