"""Pins of the CPU oracle against what the paper and mathematics fix.

* widths and sizes equal the paper's closed forms (Sections 3.2.1, 3.2.2, 3.3,
  3.4 and Table 4 for bvSD), with the bits() reading at powers of two;
* decode(encode(G)) == G for every mode on every graph with n <= 5 and on random
  graphs (round trip);
* Elias-Fano select by samples == select by a linear scan == the plain offsets;
* the DM permuter is a bijection, monotone in degree, and an isomorphism.
"""
import math

import numpy as np
import pytest

import gen
import oracle
from helpers import all_graphs, ceil_log2, csr_from_edges

ALL_MODES = [(m, o) for m in (oracle.ID_GLOBAL, oracle.ID_LOCAL, oracle.ID_LOCAL_GAP)
             for o in (oracle.OFF_PACKED, oracle.OFF_EF)]


def rows(rp, col):
    return [list(col[rp[v]:rp[v + 1]]) for v in range(len(rp) - 1)]


# ---------------------------------------------------------------- widths
def test_bits_definition():
    for x in range(0, 5000):
        assert oracle.bits(x) == (0 if x == 0 else math.floor(math.log2(x)) + 1)
    for k in range(1, 64):
        assert oracle.bits((1 << k) - 1) == k
        assert oracle.bits(1 << k) == k + 1


@pytest.mark.parametrize("scale", [3, 8, 11])
def test_global_size_closed_form(scale):
    g = gen.rmat(scale, 8, seed=scale)
    e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=oracle.ID_GLOBAL)
    # Section 3.2.1: |A| = 2m ceil(log n)
    assert e.s == ceil_log2(g.n)
    assert e.bits_A == g.arcs * ceil_log2(g.n)
    # Section 3.4: each offset in ceil(log 2m) bits (bits(2m) at the sentinel)
    assert e.w_O == ceil_log2(g.arcs + 1)
    if g.arcs & (g.arcs - 1):
        assert e.w_O == ceil_log2(g.arcs)
    assert e.bits_O == (g.n + 1) * e.w_O


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 9, 16, 17, 1000, 1024, 1025])
def test_global_width_at_power_of_two_boundaries(n):
    edges = [(i, i + 1) for i in range(n - 1)]
    rp, col, _ = csr_from_edges(n, edges)
    e = oracle.encode(n, rp, col)
    assert e.s == ceil_log2(n)
    assert e.bits_A == 2 * (n - 1) * ceil_log2(n)


def test_weighted_size_closed_form():
    g = gen.rmat(9, 8, seed=3, weighted=True)
    e = oracle.encode(g.n, g.row_ptr, g.col, g.weights)
    maxw = int(g.weights.max())
    # Section 3.3: |A| = 2m (ceil(log n) + ceil(log maxW)); bits(maxW) when maxW = 2^k
    assert e.omega == ceil_log2(maxw + 1)
    assert e.bits_A == g.arcs * (ceil_log2(g.n) + ceil_log2(maxw + 1))
    e8 = oracle.encode(g.n, g.row_ptr, g.col, g.weights, weight_bits=8)
    assert e8.omega == 8 and e8.bits_A == g.arcs * (ceil_log2(g.n) + 8)
    with pytest.raises(oracle.OracleError):
        oracle.encode(g.n, g.row_ptr, g.col, g.weights, weight_bits=4)


def test_local_size_closed_form():
    g = gen.rmat(10, 8, seed=4)
    e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=oracle.ID_LOCAL)
    H = e.H
    assert H == ceil_log2(e.s + 1)
    total = 0
    for v, r in enumerate(rows(g.row_ptr, g.col)):
        d = len(r)
        if d == 0:
            total += H
            continue
        mx = int(r[-1])
        wv = max(1, ceil_log2(mx + 1))
        # Section 3.2.2: d_v ceil(log maxN_v) bits; equal to bits(maxN_v) off powers of two
        if mx >= 2 and mx & (mx - 1):
            assert wv == ceil_log2(mx)
        # the fixed header is at least the paper's lower bound ceil(log log maxN_v)
        if mx >= 2:
            assert H >= ceil_log2(max(1, ceil_log2(mx)))
        total += d * wv + H
        assert int(e.x[v + 1] - e.x[v]) == d * wv + H
    assert e.bits_A == total


def test_local_gap_size_closed_form():
    g = gen.rmat(10, 8, seed=5)
    e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=oracle.ID_LOCAL_GAP)
    total = 0
    for v, r in enumerate(rows(g.row_ptr, g.col)):
        d = len(r)
        if d >= 2:
            gmax = max(int(r[i]) - int(r[i - 1]) for i in range(1, d))
            gw = max(1, ceil_log2(gmax + 1))
        else:
            gw = 0
        # Section 3.6: the largest difference sets the width of all differences
        ln = e.H + (e.s if d >= 1 else 0) + max(0, d - 1) * gw
        assert int(e.x[v + 1] - e.x[v]) == ln
        total += ln
    assert e.bits_A == total


def test_ef_size_formula():
    g = gen.rmat(12, 16, seed=6)
    for mode in (oracle.ID_GLOBAL, oracle.ID_LOCAL_GAP):
        e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=mode, off_mode=oracle.OFF_EF)
        N, U = g.n + 1, int(e.x[-1])
        assert e.ef_N == N and e.ef_U == U
        assert e.ef_l == (0 if U // N == 0 else int(math.floor(math.log2(U // N))))
        exact = N * e.ef_l + N + (U >> e.ef_l) + 1
        assert e.ef_low_bits + e.ef_high_bits == exact
        # Table 4 (bvSD): about n (2 + log(U / n)) bits
        approx = N * (2 + math.log2(U / N))
        assert abs(exact - approx) <= N + 2


# ---------------------------------------------------------------- round trips
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_roundtrip_exhaustive_tiny(n):
    for edges in all_graphs(n):
        rp, col, _ = csr_from_edges(n, edges)
        want = rows(rp, col)
        for mode, off in ALL_MODES:
            for relabel in (False, True):
                e = oracle.encode(n, rp, col, id_mode=mode, off_mode=off, relabel=relabel, sample=512)
                for v in range(n):
                    assert list(e.neighbors(v)) == want[v]
                    assert e.offset(v) == int(e.x[v])
                assert e.offset(n) == int(e.x[n])


@pytest.mark.parametrize("seed", range(4))
def test_roundtrip_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 300))
    m = int(rng.integers(0, 4 * n))
    edges = rng.integers(0, n, size=(m, 2))
    w = rng.integers(1, 256, size=m)
    rp, col, wt = csr_from_edges(n, edges.tolist(), w.tolist())
    want = rows(rp, col)
    wrows = [list(wt[rp[v]:rp[v + 1]]) for v in range(n)]
    for mode, off in ALL_MODES:
        for relabel in (False, True):
            e = oracle.encode(n, rp, col, id_mode=mode, off_mode=off, relabel=relabel, sample=64)
            for v in range(n):
                assert list(e.neighbors(v)) == want[v]
                assert e.degree(e.perm[v] if relabel else v) == len(want[v])
    for relabel in (False, True):
        e = oracle.encode(n, rp, col, wt, relabel=relabel, off_mode=oracle.OFF_EF, sample=64)
        for v in range(n):
            ids, ws = e.neighbors(v, with_weights=True)
            assert list(ids) == want[v] and list(ws) == wrows[v]


def test_roundtrip_rmat_with_width_straddles():
    # s + omega = 35 bits records straddle 64-bit words at every offset mod 64
    g = gen.rmat(11, 16, seed=7, weighted=True)
    e = oracle.encode(g.n, g.row_ptr, g.col, g.weights, weight_bits=24)
    assert e.r == 11 + 24
    for v in range(0, g.n, 7):
        ids, ws = e.neighbors(v, with_weights=True)
        lo, hi = g.row_ptr[v], g.row_ptr[v + 1]
        assert np.array_equal(ids, g.col[lo:hi]) and np.array_equal(ws, g.weights[lo:hi])


def test_unsupported_and_invalid():
    rp, col, _ = csr_from_edges(3, [(0, 1)])
    with pytest.raises(oracle.OracleError) as ei:
        oracle.encode(3, rp, col, np.array([1, 1], dtype=np.uint32), id_mode=oracle.ID_LOCAL)
    assert ei.value.code == 6
    with pytest.raises(oracle.OracleError):  # a row out of order
        oracle.encode(3, np.array([0, 2, 2, 2], dtype=np.uint64), np.array([2, 1], dtype=np.uint32))
    with pytest.raises(oracle.OracleError):
        oracle.encode(3, rp, np.array([3, 0], dtype=np.uint32))  # id out of range
    with pytest.raises(oracle.OracleError):
        oracle.encode(3, np.array([0, 2, 2, 2], dtype=np.uint64), np.array([1, 1], dtype=np.uint32))


# ---------------------------------------------------------------- Elias-Fano
def test_ef_select_samples_and_linear():
    g = gen.rmat(10, 4, seed=8)
    for sample in (32, 512):
        e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=oracle.ID_LOCAL_GAP, off_mode=oracle.OFF_EF,
                          sample=sample)
        for j in list(range(0, g.n + 1, 13)) + [g.n]:
            p = e.ef_select(j)
            assert p == e.ef_select_linear(j)
            # select(j) - j recovers the high part, the low bits the rest (Section 4.3)
            assert (p - j) == int(e.x[j]) >> e.ef_l
            assert e.offset(j) == int(e.x[j])
        for k in range(e.n_samples):
            assert int(e.samples[k]) == e.ef_select_linear(k * sample)


# ---------------------------------------------------------------- DM permuter
def test_dm_bijection_monotone_isomorphism():
    g = gen.rmat(10, 8, seed=9)
    e = oracle.encode(g.n, g.row_ptr, g.col, id_mode=oracle.ID_LOCAL_GAP, relabel=True)
    perm, inv = e.perm.astype(np.int64), e.inv_perm.astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(g.n))
    assert np.array_equal(perm[inv], np.arange(g.n))
    deg = g.degrees()
    dn = deg[inv]
    assert np.all(np.diff(dn) <= 0)  # higher degree -> smaller label
    ties = np.where(np.diff(dn) == 0)[0]
    assert np.all(inv[ties] < inv[ties + 1])  # ties by original ID
    # stored rows are the relabeled neighborhoods
    for v in range(0, g.n, 5):
        want = sorted(int(perm[u]) for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]])
        assert list(e.decode_raw(int(perm[v]))) == want


# ---------------------------------------------------------------- oracle pieces for large graphs
def test_ef_build_and_global_words_match_full_encode():
    g = gen.rmat(11, 8, seed=12, weighted=True)
    e = oracle.encode(g.n, g.row_ptr, g.col, g.weights, id_mode=oracle.ID_GLOBAL, off_mode=oracle.OFF_EF,
                      sample=64, weight_bits=9)
    low, high, smp, l = oracle.ef_build(g.row_ptr, sample=64)
    assert l == e.ef_l
    assert np.array_equal(low, e.ef_low) and np.array_equal(high, e.ef_high) and np.array_equal(smp, e.samples)
    used = (e.bits_A + 63) // 64
    for w0, w1 in [(0, 5), (3, 70), (used - 9, used), (0, used)]:
        got = oracle.global_words(g.col, g.weights, e.s, e.omega, w0, w1)
        assert np.array_equal(got, e.A[w0:w1])


def test_pagerank_threads_identical():
    g = gen.rmat(10, 8, seed=13)
    a = oracle.pagerank(g.n, g.row_ptr, g.col, 0.85, 7)
    b = oracle.pagerank(g.n, g.row_ptr, g.col, 0.85, 7, threads=4)
    assert np.array_equal(a, b)
