"""lg_pagerank_noalloc: the PageRank entry point for callers that cannot
allocate device memory (their memory belongs to another allocator or a fixed
budget).  It is called here through the C ABI and must give the results of
lg_pagerank, on two calls in a row (the second reuses the library's scratch
array as the first left it).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import paper_2010_15879_gb300 as lg

pytestmark = pytest.mark.gpu

RTOL = 1e-4  # the PageRank tolerance of the parity tests


def _cuda(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


def _call(lib, g, damping, iters, out, personalize=None):
    ps = None if personalize is None else ctypes.byref(ctypes.c_uint32(personalize))
    return lib.lg_pagerank_noalloc(g.handle, ctypes.c_float(damping), iters, ps, out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("mode,off,relabel", [(lg.LG_ID_LOCAL_GAP, lg.LG_OFF_EF, True),
                                              (lg.LG_ID_GLOBAL, lg.LG_OFF_PACKED, False)])
def test_noalloc_matches_pagerank_twice(mode, off, relabel):
    lib = lg.load(auto_build=True)
    g0 = gen.rmat_s16_ef16()
    g = lg.lg_encode(_cuda(g0.row_ptr, np.int64), _cuda(g0.col, np.int32), id_mode=mode, off_mode=off,
                     relabel=relabel)
    for personalize in (None, int(gen.sources(g0, 1, seed=3)[0])):
        want = lg.lg_pagerank(g, 0.85, 20, personalize=personalize).cpu().numpy()
        for _ in range(2):
            out = torch.full((g0.n,), -1.0, dtype=torch.float32, device="cuda")
            assert _call(lib, g, 0.85, 20, out, personalize) == 0, lg.lg_last_error()
            got = out.cpu().numpy()
            nz = want > 0
            assert np.all(np.abs(got[nz] - want[nz]) <= RTOL * want[nz])
            assert np.all(got[~nz] == want[~nz])


def test_noalloc_rejects_graphs_beyond_its_limit():
    lib = lg.load(auto_build=True)
    n = (1 << 20) + 1
    rp = np.zeros(n + 1, dtype=np.uint64)
    rp[1:] = 2
    rp[0] = 0
    rp[1] = 1  # one edge 0 - n-1
    rp[2:] = 1
    rp[-1] = 2
    col = np.array([n - 1, 0], dtype=np.uint32)
    g = lg.lg_encode(_cuda(rp, np.int64), _cuda(col, np.int32))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    assert _call(lib, g, 0.85, 5, out) == 4  # LG_ERANGE
    assert "at most 1048576 vertices" in lg.lg_last_error()
