"""GPU: the library's device memory pool (graph arrays and call scratch).

Freed graphs return their blocks to the pool, which keeps them mapped for the
next encode; lg_pool_trim hands them back to the system.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2010_15879_gb300 as lg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lg.load(auto_build=True)
    torch.cuda.init()


def _encode(g0):
    rp = torch.from_numpy(g0.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy(g0.col.view(np.int32)).cuda()
    return lg.lg_encode(rp, col, None, id_mode=lg.LG_ID_LOCAL_GAP, off_mode=lg.LG_OFF_EF, relabel=1)


def test_pool_reuses_and_trims():
    g0 = gen.rmat(16, 16, seed=21)
    dev = torch.cuda.current_device()
    g = _encode(g0)
    reserved1, used1 = lg.lg_pool_usage(dev)
    st = lg.lg_stats_get(g)
    assert used1 >= st["bytes_A"] > 0 and reserved1 >= used1
    lg.lg_free(g)
    g.free()  # a second release is a no-op, and so is the destructor
    with pytest.raises(lg.LgError):
        lg.lg_stats_get(g)
    reserved2, used2 = lg.lg_pool_usage(dev)
    assert used2 <= used1 - st["bytes_A"]
    assert reserved2 >= used1  # kept mapped
    # a second encode of the same graph fits in what the pool holds
    g = _encode(g0)
    reserved3, _ = lg.lg_pool_usage(dev)
    assert reserved3 <= reserved2 + (reserved2 >> 4)
    ranks = lg.lg_pagerank(g, 0.85, 3).cpu().numpy().astype(np.float64)
    want = oracle.pagerank(g0.n, g0.row_ptr, g0.col, 0.85, 3, -1)
    nz = want > 0
    assert np.max(np.abs(ranks[nz] - want[nz]) / want[nz]) <= 1e-4
    lg.lg_free(g)
    lg.lg_pool_trim(dev, 0)
    reserved4, used4 = lg.lg_pool_usage(dev)
    assert reserved4 < reserved3 and reserved4 - used4 <= (32 << 20)


def test_pool_bad_device():
    with pytest.raises(lg.LgError):
        lg.lg_pool_usage(-1)
    with pytest.raises(lg.LgError):
        lg.lg_pool_trim(64, 0)


def test_two_streams_host_inputs_and_async_free():
    """Steps alternating between two streams (host CSR copied on the call's
    stream, arrays released in stream order) give the default-stream results."""
    g0 = gen.rmat(14, 16, seed=23)
    rp_p = torch.from_numpy(g0.row_ptr.view(np.int64)).pin_memory()
    col_p = torch.from_numpy(g0.col.view(np.int32)).pin_memory()
    src = np.array([0, 5, 77, 1000], dtype=np.uint32)
    opts = dict(id_mode=lg.LG_ID_LOCAL_GAP, off_mode=lg.LG_OFF_EF, relabel=1)
    g = lg.lg_encode(rp_p, col_p, **opts)
    want_d = lg.lg_bfs(g, src).cpu().numpy()
    want_r = lg.lg_pagerank(g, 0.85, 5).cpu().numpy()
    lg.lg_free(g)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for k in range(4):
        s = streams[k & 1]
        g = lg.lg_encode(rp_p, col_p, stream=s, **opts)
        d = lg.lg_bfs(g, torch.from_numpy(src.view(np.int32)), stream=s)
        r = lg.lg_pagerank(g, 0.85, 5, stream=s)
        with torch.cuda.stream(s):
            dh = torch.empty(d.shape, dtype=d.dtype).pin_memory()
            rh = torch.empty(r.shape, dtype=r.dtype).pin_memory()
            dh.copy_(d, non_blocking=True)
            rh.copy_(r, non_blocking=True)
        lg.lg_free_async(g, s)
        outs.append((s, dh, rh))
    torch.cuda.synchronize()
    for _, dh, rh in outs:
        assert np.array_equal(dh.numpy(), want_d)
        assert np.array_equal(rh.numpy(), want_r)
