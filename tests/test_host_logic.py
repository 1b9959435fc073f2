"""CPU tests of host logic around the GPU path: the binding's stream routing
and the bench's rule for using committed ncu traffic figures."""
import contextlib
import json
import os

import pytest

import bench
import paper_2010_15879_gb300 as lg


class _FakeStream:
    cuda_stream = 1234


def test_on_stream_makes_the_call_stream_current(monkeypatch):
    entered = []

    @contextlib.contextmanager
    def fake_stream_ctx(s):
        entered.append(s)
        yield

    monkeypatch.setattr(lg.torch.cuda, "stream", fake_stream_ctx)

    @lg._on_stream
    def call(a, b=0, *, stream=None):
        return (a, b, len(entered))

    s = _FakeStream()
    assert call(1, b=2) == (1, 2, 0)  # no stream: no context
    assert call(1, stream=s) == (1, 0, 1) and entered == [s]
    assert call(3, 4, stream=s) == (3, 4, 2) and entered == [s, s]


def test_on_stream_wraps_every_stream_taking_entry_point():
    for name in ("lg_encode", "lg_neighbors", "lg_decode", "lg_bfs", "lg_sssp", "lg_pagerank",
                 "lg_pagerank_noalloc", "lg_batch_create", "lg_batch_run", "lg_batch_status"):
        fn = getattr(lg, name)
        assert fn.__wrapped__ is not None, name  # functools.wraps of _on_stream


def test_traffic_used_only_for_the_current_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2010_15879_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "lg_traverse.cuh").write_text("kernel v1")
    (csrc / "lg_device.cuh").write_text("device v1")
    (csrc / "lg_batch.cu").write_text("batch v1")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_hash("community")
    assert sha != bench.kernel_source_hash("batch")
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"community": {"source_sha": sha, "dram_bytes_per_launch": 123},
         "batch": {"source_sha": "stale", "dram_bytes_per_launch": 456}}))
    assert bench.ncu_traffic("community") == 123
    assert bench.ncu_traffic("batch") is None  # taken on another source
    (csrc / "lg_traverse.cuh").write_text("kernel v2")
    assert bench.ncu_traffic("community") is None  # the kernel changed since
    os.remove(tmp_path / "profiles" / "traffic.json")
    assert bench.ncu_traffic("community") is None
