"""CPU tests of the benchmark's bookkeeping: the per-arm comparison it
reports (GTEPS ratios against the 32-bit CSR arms, compressed bytes against
the weighted and unweighted CSR) and the serving latency summary."""
import types

import numpy as np
import pytest

import bench


def _wl(n, arcs, weighted, T=20, S=16):
    return types.SimpleNamespace(n=n, arcs=arcs, T=T, S=S, desc="test graph",
                                 w_d=object() if weighted else None)


def _arm(ms_step, enc, bfs, pr_total, steps=4):
    return {"ms": ms_step * steps, "enc": [enc] * steps, "bfs": [bfs] * steps, "pr": [pr_total] * steps}


def _arms(stats, with_dm=True):
    lg = dict(_arm(100.0, 30.0, 10.0, 60.0), stats=stats)
    return {"lg": lg, "csr": _arm(150.0, 5.0, 20.0, 120.0),
            "csr_dm": _arm(90.0, 25.0, 8.0, 54.0) if with_dm else None,
            "te_step": 4e9, "te_bfs": 1e9, "te_pr": 2e9}


def test_ratios_are_time_ratios_of_the_same_work():
    n, arcs = 1000, 16000
    st = {"bits_A": arcs * 10, "bits_O": (n + 1) * 14, "bits_per_arc": 10.9, "bytes_total": 0,
          "s": 10, "omega": 0, "id_mode": 0}
    d = bench.arms_detail(_wl(n, arcs, False), _arms(st))
    assert d["step_ms"] == pytest.approx(100.0)
    assert d["value_gteps"] == pytest.approx(4e9 / 0.1 / 1e9)
    assert d["pr_ms_per_iter"] == pytest.approx(60.0 / 20)
    # the same traversed edges on both arms: GTEPS ratio = inverse time ratio
    assert d["bfs_gteps_vs_csr32"] == pytest.approx(20.0 / 10.0)
    assert d["pr_gteps_vs_csr32"] == pytest.approx(120.0 / 60.0)
    assert d["csr32_dm_order"]["bfs_gteps_vs"] == pytest.approx(8.0 / 10.0)
    assert d["csr32_dm_order"]["pr_gteps_vs"] == pytest.approx(54.0 / 60.0)
    assert d["csr32"]["pr_gteps"] == pytest.approx(2e9 / 0.120 / 1e9)
    # unweighted: compressed bytes against 4 B per arc + 8 B per offset
    assert d["bytes_vs_csr32"] == pytest.approx((arcs * 10 + (n + 1) * 14) / 8 / (4 * arcs + 8 * (n + 1)))
    assert "bytes_vs_weighted_csr32" not in d


def test_weighted_bytes_against_both_csr_forms():
    n, arcs, s, om = 1 << 10, 1 << 14, 10, 8
    st = {"bits_A": arcs * (s + om), "bits_O": (n + 1) * 12, "bits_per_arc": 18.8, "bytes_total": 0,
          "s": s, "omega": om, "id_mode": 0}
    d = bench.arms_detail(_wl(n, arcs, True), _arms(st, with_dm=False))
    assert d["csr32_dm_order"] is None
    # 35-bit-style records against 32-bit IDs + 32-bit weights
    assert d["bytes_vs_weighted_csr32"] == pytest.approx((arcs * (s + om) + (n + 1) * 12) / 8 /
                                                         (8 * arcs + 8 * (n + 1)))
    # the same IDs without their weights against the unweighted CSR-32
    assert d["bytes_unweighted_vs_csr32"] == pytest.approx((arcs * s + (n + 1) * 12) / 8 /
                                                           (4 * arcs + 8 * (n + 1)))
    st_local = dict(st, id_mode=2)
    assert bench.arms_detail(_wl(n, arcs, True), _arms(st_local))["bytes_unweighted_vs_csr32"] is None


def test_latency_summary_per_kind():
    rng = np.random.default_rng(3)
    kinds = rng.integers(0, 3, size=10000)
    lat_ns = ((kinds + 1) * 1_000_000 + rng.integers(0, 1000, size=10000)).astype(np.int64)
    s = bench.latency_summary(lat_ns, kinds)
    assert s["p50_ms"] == pytest.approx(np.percentile(lat_ns / 1e6, 50))
    assert s["p99_ms"] == pytest.approx(np.percentile(lat_ns / 1e6, 99))
    for k, name in enumerate(("lookup", "bfs", "ppr")):
        assert k + 1 <= s[name]["p50_ms"] < k + 1.001
    only_lookups = bench.latency_summary(lat_ns[kinds == 0], kinds[kinds == 0])
    assert "bfs" not in only_lookups and "ppr" not in only_lookups


def test_host_cores_is_the_affinity_count():
    assert 1 <= bench.host_cores()
