"""GB300 Log(Graph): Python binding of liblg.so.

The functions here carry the names of the C ABI in ``include/lg.h`` and do
argument marshalling only: every step of the encoder and of the graph kernels
runs in the CUDA library.  PyTorch provides device memory and streams.  There is
no CPU fallback: if liblg.so is missing or no GPU is present, the calls raise.

Quick use::

    import torch, paper_2010_15879_gb300 as lg
    g = lg.lg_encode(row_ptr_cuda_u64, col_cuda_u32, id_mode=lg.LG_ID_LOCAL_GAP,
                     off_mode=lg.LG_OFF_EF, relabel=True)
    depths = lg.lg_bfs(g, sources_cuda_u32)          # (S, n) uint32 as int32
    ranks = lg.lg_pagerank(g, 0.85, 20)              # (n,) float32
"""
from __future__ import annotations

import ctypes
import functools
import inspect
import os
import threading
from typing import Optional

import numpy as np
import torch

from ._build import LIB, build, is_stale

__all__ = [
    "LG_ID_GLOBAL", "LG_ID_LOCAL", "LG_ID_LOCAL_GAP", "LG_ID_CSR32", "LG_OFF_PACKED", "LG_OFF_EF",
    "LG_RELABEL_NONE", "LG_RELABEL_DM", "LG_RELABEL_GREEDY",
    "LgError", "LogGraph", "build", "load", "lg_encode", "lg_stats_get", "lg_arrays_get", "lg_arrays_device",
    "lg_neighbors",
    "lg_bfs", "lg_sssp", "lg_pagerank", "lg_pagerank_noalloc", "lg_free", "lg_last_error", "lg_kernel_launches",
    "lg_decode", "lg_free_async", "lg_pool_trim", "lg_pool_usage", "lg_probe_gather",
    "LgBatch", "lg_batch_create", "lg_batch_run", "lg_batch_status", "lg_batch_info_get", "lg_batch_free",
    "LG_BATCH_FLAG_DROP_MEMBER",
    "LG_REQ_NEIGHBORS", "LG_REQ_BFS", "LG_REQ_PPR", "LgServer", "lg_server_create", "lg_server_submit",
    "lg_server_wait", "lg_server_release", "lg_server_stats_get", "lg_server_replay", "lg_server_destroy",
    "lg_server_engine_time",
]

LG_ID_GLOBAL, LG_ID_LOCAL, LG_ID_LOCAL_GAP, LG_ID_CSR32 = 0, 1, 2, 3
LG_OFF_PACKED, LG_OFF_EF = 0, 1
LG_RELABEL_NONE, LG_RELABEL_DM, LG_RELABEL_GREEDY = 0, 1, 2
LG_FLAG_CHECK_SYMMETRIC = 1
LG_BATCH_FLAG_DROP_MEMBER = 1
LG_REQ_NEIGHBORS, LG_REQ_BFS, LG_REQ_PPR = 0, 1, 2
STATUS = {0: "LG_OK", 1: "LG_EINVAL", 2: "LG_ENOMEM", 3: "LG_ECUDA", 4: "LG_ERANGE", 5: "LG_ETIMEOUT",
          6: "LG_EUNSUPPORTED"}

_u64, _u32, _i32, _f32, _dbl, _vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_double, ctypes.c_void_p)


class _Opts(ctypes.Structure):
    _fields_ = [("id_mode", _u32), ("off_mode", _u32), ("relabel", _u32), ("select_sample", _u32),
                ("weight_bits", _u32), ("flags", _u32)]


class _Stats(ctypes.Structure):
    _fields_ = [("n", _u64), ("arcs", _u64), ("bits_A", _u64), ("bits_O", _u64), ("bytes_A", _u64),
                ("bytes_O", _u64), ("bytes_perm", _u64), ("bytes_total", _u64), ("max_degree", _u64),
                ("id_mode", _u32), ("off_mode", _u32), ("relabel", _u32), ("weighted", _u32), ("s", _u32),
                ("H", _u32), ("omega", _u32), ("w_O", _u32), ("ef_l", _u32), ("select_sample", _u32),
                ("bits_per_arc", _dbl), ("bytes_schedule", _u64)]


class _Arrays(ctypes.Structure):
    _fields_ = [("A", _vp), ("words_A", _u64), ("O", _vp), ("words_O", _u64), ("ef_low", _vp),
                ("words_ef_low", _u64), ("ef_high", _vp), ("words_ef_high", _u64), ("ef_samples", _vp),
                ("words_ef_samples", _u64), ("perm", _vp), ("inv_perm", _vp)]


class _BatchOpts(ctypes.Structure):
    _fields_ = [("autotune", _u32), ("lanes", _u32), ("tile_arcs", _u64), ("wait_limit_us", _u32),
                ("flags", _u32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("count", _u32), ("V", _u64), ("arcs", _u64), ("A", _vp), ("words_A", _u64), ("O", _vp),
                ("words_O", _u64), ("graphs", _vp), ("n_items", _u32), ("grid", _u32), ("threads", _u32),
                ("tile_arcs", _u64), ("teams", _u32), ("max_team", _u32), ("bits_total", _u64),
                ("launches", _u64), ("graphs_by_lanes", _u32 * 4)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("device_bytes", _u64), ("host_bytes", _u64), ("bfs_slots", _u32), ("ppr_slots", _u32),
                ("nbr_batch_vertices", _u32), ("ppr_iters", _u32)]


class _Request(ctypes.Structure):
    _fields_ = [("kind", _u32), ("graph", _u32), ("source", _u32), ("iters", _u32), ("damping", _f32),
                ("count", _u32), ("vertices", _vp), ("user", _u64)]


class _Result(ctypes.Structure):
    _fields_ = [("ticket", _u64), ("user", _u64), ("kind", _u32), ("graph", _u32), ("status", _i32),
                ("data", _vp), ("bytes", _u64), ("count", _u64), ("t_submit_ns", _u64), ("t_admit_ns", _u64),
                ("t_done_ns", _u64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(k, _u64) for k in ("submitted", "completed", "failed")] + [("by_kind", _u64 * 3)] + [
        (k, _u64) for k in ("bfs_levels", "bfs_joins", "bfs_joins_running", "bfs_max_active", "ppr_iterations",
                            "ppr_joins", "ppr_joins_running", "ppr_max_active", "nbr_batches", "nbr_max_batch",
                            "admission_waits", "device_bytes", "device_used", "device_peak", "host_bytes",
                            "host_used", "host_peak")]


class _ReplayStats(ctypes.Structure):
    _fields_ = [("completed", _u64), ("failed", _u64), ("makespan_ns", _u64)]


class LgError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what} -> {STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(auto_build: bool = False):
    """Load liblg.so (building it first only when ``auto_build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if auto_build and is_stale():
            build()
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is not built: run paper_2010_15879_gb300.build() (nvcc, sm_103a)")
        h = ctypes.CDLL(LIB)
        h.lg_encode.argtypes = [_vp, _vp, _vp, _u64, _u64, ctypes.POINTER(_Opts), _vp, ctypes.POINTER(_vp)]
        h.lg_stats_get.argtypes = [_vp, ctypes.POINTER(_Stats)]
        h.lg_arrays_get.argtypes = [_vp, ctypes.POINTER(_Arrays)]
        h.lg_neighbors.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp, _u64, _vp]
        h.lg_bfs.argtypes = [_vp, _vp, _u32, _vp, _vp]
        h.lg_sssp.argtypes = [_vp, _u32, _u64, _vp, _vp]
        h.lg_pagerank.argtypes = [_vp, _f32, _u32, ctypes.POINTER(_u32), _vp, _vp]
        h.lg_pagerank_noalloc.argtypes = [_vp, _f32, _u32, ctypes.POINTER(_u32), _vp, _vp]
        h.lg_free.argtypes = [_vp]
        h.lg_decode.argtypes = [_vp, _vp, _vp, _vp, _u64, _vp]
        h.lg_decode.restype = ctypes.c_int
        h.lg_free_async.argtypes = [_vp, _vp]
        h.lg_free_async.restype = ctypes.c_int
        h.lg_pool_trim.argtypes = [ctypes.c_int, _u64]
        h.lg_pool_trim.restype = ctypes.c_int
        h.lg_pool_usage.argtypes = [ctypes.c_int, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
        h.lg_pool_usage.restype = ctypes.c_int
        h.lg_free.restype = None
        h.lg_last_error.restype = ctypes.c_char_p
        h.lg_probe_gather.argtypes = [_vp, _u64, _vp, _u64, _vp, _vp]
        h.lg_probe_gather.restype = _i32
        h.lg_kernel_launches.argtypes = []
        h.lg_kernel_launches.restype = _u64
        h.lg_batch_create.argtypes = [_vp, _vp, _vp, _u32, _u64, _u64, ctypes.POINTER(_BatchOpts), _vp,
                                      ctypes.POINTER(_vp)]
        h.lg_batch_run.argtypes = [_vp, _f32, _u32, _vp, _vp, _vp]
        h.lg_batch_status.argtypes = [_vp, _vp]
        h.lg_batch_info_get.argtypes = [_vp, ctypes.POINTER(_BatchInfo)]
        h.lg_batch_free.argtypes = [_vp]
        h.lg_batch_free.restype = None
        h.lg_server_create.argtypes = [ctypes.POINTER(_vp), _u32, ctypes.POINTER(_ServerOpts), ctypes.POINTER(_vp)]
        h.lg_server_submit.argtypes = [_vp, ctypes.POINTER(_Request), ctypes.POINTER(_u64)]
        h.lg_server_wait.argtypes = [_vp, ctypes.POINTER(_Result), _u32, ctypes.POINTER(_u32), _u32]
        h.lg_server_release.argtypes = [_vp, _u64]
        h.lg_server_stats_get.argtypes = [_vp, ctypes.POINTER(_ServerStats)]
        h.lg_server_replay.argtypes = [_vp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                       ctypes.POINTER(_ReplayStats)]
        h.lg_server_engine_time.argtypes = [_vp, _u32, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
        h.lg_server_destroy.argtypes = [_vp]
        h.lg_server_destroy.restype = None
        for f in ("lg_encode", "lg_stats_get", "lg_arrays_get", "lg_neighbors", "lg_bfs", "lg_pagerank",
                  "lg_pagerank_noalloc", "lg_sssp", "lg_batch_create", "lg_batch_run", "lg_batch_status",
                  "lg_batch_info_get", "lg_server_create", "lg_server_submit", "lg_server_wait",
                  "lg_server_release", "lg_server_stats_get", "lg_server_replay", "lg_server_engine_time"):
            getattr(h, f).restype = _i32
        _lib = h
    return _lib


def lg_last_error() -> str:
    return load().lg_last_error().decode()


def lg_kernel_launches() -> int:
    """Kernels launched by liblg.so in this process so far."""
    return int(load().lg_kernel_launches())


PROBE_THREADS = 152 * 8 * 256  # threads of one lg_probe_gather launch (at most)


def lg_probe_gather(idx: torch.Tensor, table: torch.Tensor, out: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    """lg_probe_gather: table[idx[i]] gathered for every i (idx int32 holding
    uint32 values < table.numel(), table float32, both on the device); returns
    the per-thread partial sums."""
    if idx.dtype != torch.int32 or table.dtype != torch.float32 or not (idx.is_cuda and table.is_cuda):
        raise TypeError("lg_probe_gather: idx must be int32 and table float32, on the device")
    if out is None:
        out = torch.empty(max(1, min(idx.numel(), PROBE_THREADS)), dtype=torch.float32, device=idx.device)
    _check(load().lg_probe_gather(idx.data_ptr(), idx.numel(), table.data_ptr(), table.numel(), out.data_ptr(),
                                  _stream(stream)), "lg_probe_gather")
    return out


def lg_pool_trim(device: int = 0, keep_bytes: int = 0) -> None:
    """Release pooled device memory of `device` down to keep_bytes reserved."""
    _check(load().lg_pool_trim(int(device), int(keep_bytes)), "lg_pool_trim")


def lg_pool_usage(device: int = 0) -> tuple:
    """(reserved, used) bytes of the library's device memory pool."""
    r, u = _u64(0), _u64(0)
    _check(load().lg_pool_usage(int(device), ctypes.byref(r), ctypes.byref(u)), "lg_pool_usage")
    return int(r.value), int(u.value)


def _check(status: int, what: str):
    if status != 0:
        raise LgError(status, what, lg_last_error())


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str, stream=None) -> torch.Tensor:
    """Device-resident contiguous tensor of the given dtype (host tensors are
    copied, in order on `stream` when one is given)."""
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.ascontiguousarray(t))
    if t.dtype != dtype:
        if t.element_size() != torch.empty(0, dtype=dtype).element_size():
            raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
        t = t.view(dtype)
    if not t.is_cuda:
        if stream is not None:
            with torch.cuda.stream(stream):
                return t.to("cuda", non_blocking=True).contiguous()
        t = t.to("cuda", non_blocking=True)
    return t.contiguous()


def _on_stream(fn):
    """Run the call with `stream` (when given) as torch's current stream, so
    that its host copies, allocations and reads are ordered with the library's
    work on that stream."""
    sig = inspect.signature(fn)

    @functools.wraps(fn)
    def call(*args, **kwargs):
        st = sig.bind_partial(*args, **kwargs).arguments.get("stream")
        if st is None:
            return fn(*args, **kwargs)
        with torch.cuda.stream(st):
            return fn(*args, **kwargs)
    return call


class LogGraph:
    """Owner of an lg_graph handle (freed with lg_free)."""

    def __init__(self, handle: int, keepalive=()):
        self._h = _vp(handle)
        self._keep = keepalive

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        return lg_stats_get(self)

    def free(self, stream=None):
        """Release the graph (once; later calls and the destructor do nothing).
        Without a stream this waits for the device to be idle (lg_free); with
        one the arrays are released in stream order on it (lg_free_async)."""
        h, self._h = self._h, None
        if h is not None and h.value:
            if stream is None:
                load().lg_free(h)
            else:
                _check(load().lg_free_async(h, _stream(stream)), "lg_free_async")

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


@_on_stream
def lg_encode(row_ptr, col, weights=None, *, id_mode: int = LG_ID_GLOBAL, off_mode: int = LG_OFF_PACKED,
              relabel: int = 0, select_sample: int = 512, weight_bits: int = 0,
              check_symmetric: bool = False, stream=None) -> LogGraph:
    """lg_encode: build the logarithmized graph from a CSR (row_ptr uint64[n+1],
    col uint32[arcs], optional weights uint32[arcs]; int64/int32 tensors are
    reinterpreted).  Host tensors are copied to the current device first."""
    lib = load()
    rp = _dev(row_ptr, torch.int64, "row_ptr", stream)
    cl = _dev(col, torch.int32, "col", stream)
    wt = None if weights is None else _dev(weights, torch.int32, "weights", stream)
    n = rp.numel() - 1
    opts = _Opts(id_mode, off_mode, int(relabel), select_sample, weight_bits,
                 LG_FLAG_CHECK_SYMMETRIC if check_symmetric else 0)
    h = _vp()
    st = _stream(stream)
    _check(lib.lg_encode(rp.data_ptr(), cl.data_ptr() if cl.numel() else None,
                         None if wt is None else wt.data_ptr(), n, cl.numel(), ctypes.byref(opts), st,
                         ctypes.byref(h)), "lg_encode")
    return LogGraph(h.value)


def lg_free(g: LogGraph) -> None:
    """Release g's device memory; g is unusable afterwards."""
    g.free()


def lg_free_async(g: LogGraph, stream=None) -> None:
    """Release g's device memory in stream order on `stream` (default: the
    current stream) without waiting; g is unusable afterwards."""
    g.free(stream if stream is not None else torch.cuda.current_stream())


def lg_stats_get(g: LogGraph) -> dict:
    s = _Stats()
    _check(load().lg_stats_get(g.handle, ctypes.byref(s)), "lg_stats_get")
    return {k: getattr(s, k) for k, _ in _Stats._fields_}


class _DevView:
    """__cuda_array_interface__ over library-owned device memory (read-only use)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def lg_arrays_get(g: LogGraph) -> dict:
    """Host (numpy) copies of the encoded arrays: uint64 word streams (with
    padding and guard words) and the uint32 permutation if relabeled."""
    a = _Arrays()
    _check(load().lg_arrays_get(g.handle, ctypes.byref(a)), "lg_arrays_get")
    n = lg_stats_get(g)["n"]
    out = {}
    torch.cuda.synchronize()
    for name in ("A", "O", "ef_low", "ef_high", "ef_samples"):
        ptr, cnt = getattr(a, name), getattr(a, "words_" + name)
        if ptr and cnt:
            t = torch.as_tensor(_DevView(ptr, cnt, "<i8"), device="cuda")
            out[name] = t.cpu().numpy().view(np.uint64).copy()
        else:
            out[name] = np.zeros(0, dtype=np.uint64)
    for name in ("perm", "inv_perm"):
        ptr = getattr(a, name)
        if ptr:
            t = torch.as_tensor(_DevView(ptr, n, "<i4"), device="cuda")
            out[name] = t.cpu().numpy().view(np.uint32).copy()
        else:
            out[name] = np.zeros(0, dtype=np.uint32)
    return out


def lg_arrays_device(g: LogGraph) -> dict:
    """Device views of the encoded arrays, without copies: int64 tensors over
    the uint64 word streams (with padding and guard words) and int32 tensors
    over the permutation if relabeled.  The memory belongs to the library: read
    only, valid until g is freed."""
    a = _Arrays()
    _check(load().lg_arrays_get(g.handle, ctypes.byref(a)), "lg_arrays_get")
    n = lg_stats_get(g)["n"]
    out = {}
    for name in ("A", "O", "ef_low", "ef_high", "ef_samples"):
        ptr, cnt = getattr(a, name), getattr(a, "words_" + name)
        out[name] = (torch.as_tensor(_DevView(ptr, cnt, "<i8"), device="cuda") if ptr and cnt
                     else torch.zeros(0, dtype=torch.int64, device="cuda"))
    for name in ("perm", "inv_perm"):
        ptr = getattr(a, name)
        out[name] = (torch.as_tensor(_DevView(ptr, n, "<i4"), device="cuda") if ptr
                     else torch.zeros(0, dtype=torch.int32, device="cuda"))
    return out


@_on_stream
def lg_decode(g: LogGraph, with_weights: bool = False, stream=None):
    """lg_decode: the whole graph as a CSR in stored order: (row_ptr int64[n+1],
    col uint32-as-int32[arcs][, weights]); stored labels for relabeled graphs."""
    lib = load()
    st_ = lg_stats_get(g)
    n, arcs = st_["n"], st_["arcs"]
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(max(arcs, 1), dtype=torch.int32, device="cuda")
    wts = torch.empty(max(arcs, 1), dtype=torch.int32, device="cuda") if with_weights else None
    _check(lib.lg_decode(g.handle, rp.data_ptr(), col.data_ptr(), None if wts is None else wts.data_ptr(), arcs,
                         _stream(stream)), "lg_decode")
    return (rp, col[:arcs], wts[:arcs]) if with_weights else (rp, col[:arcs])


@_on_stream
def lg_neighbors(g: LogGraph, vertices, with_weights: bool = False, stream=None):
    """lg_neighbors: (offsets int64[k+1], ids uint32-as-int32[total][, weights])
    for the given original vertex IDs; each slice ascending."""
    lib = load()
    vs = _dev(vertices, torch.int32, "vertices")
    k = vs.numel()
    st = _stream(stream)
    off = torch.empty(k + 1, dtype=torch.int64, device="cuda")
    vptr = vs.data_ptr() if k else None
    rc = lib.lg_neighbors(g.handle, vptr, k, off.data_ptr(), None, None, 0, st)
    if rc not in (0, 4):
        _check(rc, "lg_neighbors")
    total = int(off[-1].item())
    ids = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    wts = torch.empty(max(total, 1), dtype=torch.int32, device="cuda") if with_weights else None
    _check(lib.lg_neighbors(g.handle, vptr, k, off.data_ptr(), ids.data_ptr(),
                            None if wts is None else wts.data_ptr(), total, st), "lg_neighbors")
    ids = ids[:total]
    return (off, ids, wts[:total]) if with_weights else (off, ids)


@_on_stream
def lg_bfs(g: LogGraph, sources, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """lg_bfs: depths (S, n) as int32 holding uint32 values (UINT32_MAX = -1:
    unreachable)."""
    lib = load()
    src = _dev(sources, torch.int32, "sources")
    S = src.numel()
    n = lg_stats_get(g)["n"]
    if out is None:
        out = torch.empty((S, n), dtype=torch.int32, device="cuda")
    _check(lib.lg_bfs(g.handle, src.data_ptr() if S else None, S, out.data_ptr(), _stream(stream)), "lg_bfs")
    return out


@_on_stream
def lg_sssp(g: LogGraph, source: int, delta: int = 0, out: Optional[torch.Tensor] = None,
            stream=None) -> torch.Tensor:
    """lg_sssp: shortest-path distances (n,) as int64 holding uint64 values
    (UINT64_MAX = -1: unreachable) from `source` on a weighted graph."""
    n = lg_stats_get(g)["n"]
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device="cuda")
    _check(load().lg_sssp(g.handle, source, delta, out.data_ptr(), _stream(stream)), "lg_sssp")
    return out


@_on_stream
def lg_pagerank_noalloc(g: LogGraph, damping: float, iters: int, out: torch.Tensor,
                        personalize: Optional[int] = None, stream=None) -> torch.Tensor:
    """lg_pagerank_noalloc: PageRank into ``out`` (n float32, on the device) for
    callers that cannot allocate device memory -- the library uses a fixed
    internal scratch array instead (graphs up to 2^20 vertices)."""
    n = lg_stats_get(g)["n"]
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float32:
        raise TypeError("lg_pagerank_noalloc: out must be a float32 CUDA tensor")
    if out.numel() < n or not out.is_contiguous():
        raise ValueError(f"lg_pagerank_noalloc: out must be contiguous with at least n = {n} elements")
    dev = torch.cuda.current_device() if stream is None else stream.device.index
    if out.device.index != dev:
        raise ValueError(f"lg_pagerank_noalloc: out is on cuda:{out.device.index}, the call runs on cuda:{dev}")
    ps = None if personalize is None else ctypes.byref(_u32(personalize))
    _check(load().lg_pagerank_noalloc(g.handle, damping, iters, ps, out.data_ptr(), _stream(stream)),
           "lg_pagerank_noalloc")
    return out


@_on_stream
def lg_pagerank(g: LogGraph, damping: float = 0.85, iters: int = 20, personalize: Optional[int] = None,
                out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """lg_pagerank: FP32 ranks (n,) indexed by original vertex ID."""
    lib = load()
    n = lg_stats_get(g)["n"]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
    ps = None if personalize is None else ctypes.byref(_u32(personalize))
    _check(lib.lg_pagerank(g.handle, damping, iters, ps, out.data_ptr(), _stream(stream)), "lg_pagerank")
    return out


# --- batches -----------------------------------------------------------------

class LgBatch:
    """Owner of an lg_batch handle and of the input it references."""

    def __init__(self, handle: int, keepalive=()):
        self._h = _vp(handle)
        self._keep = keepalive  # row_ptr / col / graph_vptr: lg_batch_run re-encodes from them

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        return lg_batch_info_get(self)

    def free(self):
        if self._h is not None and self._h.value:
            load().lg_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


@_on_stream
def lg_batch_create(graph_vptr, row_ptr, col, *, autotune: bool = True, lanes: int = 0, tile_arcs: int = 0,
                    wait_limit_us: int = 0, flags: int = 0, stream=None) -> LgBatch:
    """lg_batch_create: plan a batch of graphs given as one CSR over the batch
    vertex space (graph_vptr uint64[count+1], row_ptr uint64[V+1] global arc
    offsets, col uint32[arcs] local IDs).  The device tensors are kept alive
    by the returned object, since every run re-encodes from them."""
    lib = load()
    vp = _dev(graph_vptr, torch.int64, "graph_vptr")
    rp = _dev(row_ptr, torch.int64, "row_ptr")
    cl = _dev(col, torch.int32, "col")
    opts = _BatchOpts(int(bool(autotune)), lanes, tile_arcs, wait_limit_us, flags)
    h = _vp()
    _check(lib.lg_batch_create(vp.data_ptr(), rp.data_ptr(), cl.data_ptr() if cl.numel() else None,
                               vp.numel() - 1, rp.numel() - 1, cl.numel(), ctypes.byref(opts),
                               _stream(stream), ctypes.byref(h)), "lg_batch_create")
    return LgBatch(h.value, keepalive=(vp, rp, cl))


@_on_stream
def lg_batch_run(b: LgBatch, damping: float = 0.85, iters: int = 10, depths: Optional[torch.Tensor] = None,
                 ranks: Optional[torch.Tensor] = None, stream=None):
    """lg_batch_run: encode + BFS from each graph's vertex 0 + PageRank, one
    graph launch.  Returns (depths int32[V] holding uint32, ranks float32[V])."""
    V = b.info()["V"]
    if depths is None:
        depths = torch.empty(V, dtype=torch.int32, device="cuda")
    if ranks is None:
        ranks = torch.empty(V, dtype=torch.float32, device="cuda")
    _check(load().lg_batch_run(b.handle, damping, iters, depths.data_ptr(), ranks.data_ptr(), _stream(stream)),
           "lg_batch_run")
    return depths, ranks


@_on_stream
def lg_batch_status(b: LgBatch, stream=None) -> None:
    """lg_batch_status: synchronize and raise LgError (LG_ETIMEOUT) if a team
    barrier of the last run ran out of time."""
    _check(load().lg_batch_status(b.handle, _stream(stream)), "lg_batch_status")


def lg_batch_info_get(b: LgBatch) -> dict:
    i = _BatchInfo()
    _check(load().lg_batch_info_get(b.handle, ctypes.byref(i)), "lg_batch_info_get")
    d = {k: getattr(i, k) for k, _ in _BatchInfo._fields_}
    d["graphs_by_lanes"] = dict(zip((1, 4, 8, 32), list(i.graphs_by_lanes)))
    return d


def lg_batch_arrays(b: LgBatch) -> dict:
    """Host copies of the batch's A and O word streams and its graph table
    (structured numpy array with the fields of lg_batch_graph)."""
    i = lg_batch_info_get(b)
    torch.cuda.synchronize()
    out = {}
    for name in ("A", "O"):
        t = torch.as_tensor(_DevView(i[name], i["words_" + name], "<i8"), device="cuda")
        out[name] = t.cpu().numpy().view(np.uint64).copy()
    t = torch.as_tensor(_DevView(i["graphs"], i["count"] * 8, "<i8"), device="cuda")
    raw = t.cpu().numpy().view(np.uint64).reshape(i["count"], 8)
    dt = np.dtype([("vbase", "<u8"), ("abase", "<u8"), ("a_word", "<u8"), ("o_word", "<u8"), ("n", "<u4"),
                   ("arcs", "<u4"), ("s", "<u4"), ("w_O", "<u4"), ("lanes", "<u4"), ("team", "<u4"),
                   ("pad", "<u4", 2)])
    out["graphs"] = raw.copy().view(dt).reshape(-1)
    return out


def lg_batch_free(b: LgBatch) -> None:
    b.free()


# --- serving -----------------------------------------------------------------

def _result_arrays(r: _Result):
    """numpy copies of a result's host data."""
    if not r.data or r.status != 0:
        return None
    buf = (ctypes.c_char * r.bytes).from_address(r.data)
    raw = np.frombuffer(buf, dtype=np.uint8).copy()
    if r.kind == LG_REQ_NEIGHBORS:
        off = raw[:(r.count + 1) * 8].view(np.uint64)
        return off, raw[(r.count + 1) * 8:].view(np.uint32)
    if r.kind == LG_REQ_BFS:
        return raw.view(np.uint32)
    return raw.view(np.float32)


class LgServer:
    """Owner of an lg_server handle (and of references to its graphs)."""

    def __init__(self, handle: int, graphs):
        self._h = _vp(handle)
        self.graphs = list(graphs)

    @property
    def handle(self):
        return self._h

    def destroy(self):
        if self._h is not None and self._h.value:
            load().lg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def lg_server_create(graphs, device_bytes: int = 0, host_bytes: int = 0, bfs_slots: int = 0, ppr_slots: int = 0,
                     nbr_batch_vertices: int = 0, ppr_iters: int = 0) -> LgServer:
    """lg_server_create: serve the given LogGraph objects (kept alive by the server object)."""
    arr = (_vp * len(graphs))(*[g.handle.value for g in graphs])
    opts = _ServerOpts(device_bytes, host_bytes, bfs_slots, ppr_slots, nbr_batch_vertices, ppr_iters)
    h = _vp()
    _check(load().lg_server_create(arr, len(graphs), ctypes.byref(opts), ctypes.byref(h)), "lg_server_create")
    return LgServer(h.value, graphs)


def lg_server_submit(s: LgServer, kind: int, graph: int, source: int = 0, vertices=None, iters: int = 0,
                     damping: float = 0.0, user: int = 0) -> int:
    """lg_server_submit: returns the ticket."""
    vs = None
    if vertices is not None:
        vs = np.ascontiguousarray(vertices, dtype=np.uint32)
    q = _Request(kind, graph, source, iters, damping, 0 if vs is None else vs.size,
                 None if vs is None else vs.ctypes.data, user)
    t = _u64()
    _check(load().lg_server_submit(s.handle, ctypes.byref(q), ctypes.byref(t)), "lg_server_submit")
    return t.value


def lg_server_wait(s: LgServer, max_results: int = 64, timeout_us: int = 1000000, release: bool = True):
    """lg_server_wait: list of dicts (ticket, user, kind, graph, status, result
    arrays, timestamps); results are copied out and released unless
    ``release`` is False."""
    buf = (_Result * max_results)()
    got = _u32()
    _check(load().lg_server_wait(s.handle, buf, max_results, ctypes.byref(got), timeout_us), "lg_server_wait")
    out = []
    for i in range(got.value):
        r = buf[i]
        out.append({"ticket": r.ticket, "user": r.user, "kind": r.kind, "graph": r.graph, "status": r.status,
                    "result": _result_arrays(r), "count": r.count, "t_submit_ns": r.t_submit_ns,
                    "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns})
        if release:
            lg_server_release(s, r.ticket)
    return out


def lg_server_release(s: LgServer, ticket: int) -> None:
    _check(load().lg_server_release(s.handle, ticket), "lg_server_release")


def lg_server_stats_get(s: LgServer) -> dict:
    st = _ServerStats()
    _check(load().lg_server_stats_get(s.handle, ctypes.byref(st)), "lg_server_stats_get")
    d = {k: getattr(st, k) for k, _ in _ServerStats._fields_}
    d["by_kind"] = list(st.by_kind)
    return d


def lg_server_replay(s: LgServer, kind, graph, source, nbr_off, nbr_vertices, arrival_ns, keep=None):
    """lg_server_replay: open-loop replay of a request trace (numpy columns).
    ``keep``: optional list of numpy buffers (or None) receiving results.
    Returns (latency_ns uint64[n], stats dict)."""
    kind = np.ascontiguousarray(kind, dtype=np.uint32)
    graph = np.ascontiguousarray(graph, dtype=np.uint32)
    source = np.ascontiguousarray(source, dtype=np.uint32)
    nbr_off = np.ascontiguousarray(nbr_off, dtype=np.uint64)
    nbr_vertices = np.ascontiguousarray(nbr_vertices, dtype=np.uint32)
    arrival_ns = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
    n = kind.size
    lat = np.zeros(n, dtype=np.uint64)
    keep_arr = None
    if keep is not None:
        keep_arr = (_vp * n)(*[None if k is None else k.ctypes.data for k in keep])
    st = _ReplayStats()
    rc = load().lg_server_replay(s.handle, n, kind.ctypes.data, graph.ctypes.data, source.ctypes.data,
                                 nbr_off.ctypes.data, nbr_vertices.ctypes.data if nbr_vertices.size else None,
                                 arrival_ns.ctypes.data, keep_arr, lat.ctypes.data, ctypes.byref(st))
    _check(rc, "lg_server_replay")
    return lat, {"completed": st.completed, "failed": st.failed, "makespan_ns": st.makespan_ns}


def lg_server_engine_time(s: LgServer, graph: int, kind: int):
    """(operations run, device nanoseconds) of one engine (CUDA events on its stream)."""
    ops, ns = _u64(), _u64()
    _check(load().lg_server_engine_time(s.handle, graph, kind, ctypes.byref(ops), ctypes.byref(ns)),
           "lg_server_engine_time")
    return ops.value, ns.value


def lg_server_destroy(s: LgServer) -> None:
    s.destroy()
