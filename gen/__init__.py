"""Seeded synthetic graph inputs, shared by the CPU oracle and the CUDA path.

This package holds none of the Log(Graph) arithmetic: it draws edges with a
counter-based SplitMix64 and builds a plain symmetric CSR adjacency array
(``row_ptr`` uint64[n+1], ``col`` uint32[arcs], strictly increasing rows, no
self loops), the input of the paper's Section 2.3 ("adjacency array").

Workloads (shapes of the paper's evaluation, Section 7.1, Kronecker "sX_eY"):

* :func:`rmat` -- R-MAT/Kronecker, ``2^scale`` vertices, ``edge_factor * 2^scale``
  edges, (a, b, c) = (0.57, 0.19, 0.19), seeded label permutation.
* :func:`community` -- blocks of 1024 vertices, Zipf out-degrees, 90 % of the
  edges inside the block, then a global permutation.
* :func:`from_edges` -- an explicit edge list (small test graphs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "lggen.c")
_LIB = os.path.join(_DIR, "liblggen.so")
_GPU_SRC = os.path.join(_DIR, "lggen_gpu.cu")
_GPU_LIB = os.path.join(_DIR, "liblggen_gpu.so")
_lock = threading.Lock()
_handle = None
_gpu_handle = None


class _Csr(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("arcs", ctypes.c_uint64),
        ("row_ptr", ctypes.POINTER(ctypes.c_uint64)),
        ("col", ctypes.POINTER(ctypes.c_uint32)),
        ("w", ctypes.POINTER(ctypes.c_uint32)),
    ]


def build(force: bool = False) -> str:
    """Compile ``liblggen.so`` next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_gpu(force: bool = False) -> str:
    """Compile ``liblggen_gpu.so`` (nvcc, sm_103a) for the device-side R-MAT builder."""
    if force or not os.path.exists(_GPU_LIB) or os.path.getmtime(_GPU_LIB) < os.path.getmtime(_GPU_SRC):
        import shutil
        nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _GPU_LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                               "-shared", "-o", tmp, _GPU_SRC])
        os.replace(tmp, _GPU_LIB)
    return _GPU_LIB


def _gpu_lib():
    global _gpu_handle
    with _lock:
        if _gpu_handle is None:
            build_gpu()
            h = ctypes.CDLL(_GPU_LIB)
            u64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            h.lggen_gpu_rmat_count.argtypes = [i32, u64, dbl, dbl, dbl, u64, vp, vp, vp]
            h.lggen_gpu_rmat_scatter.argtypes = [i32, u64, dbl, dbl, dbl, u64, vp, vp, vp, vp]
            h.lggen_gpu_weights.argtypes = [vp, vp, u64, u64, vp, vp]
            h.lggen_gpu_batch_edges.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.c_uint32, dbl, dbl, dbl, vp,
                                                vp, vp]
            for f in (h.lggen_gpu_rmat_count, h.lggen_gpu_rmat_scatter, h.lggen_gpu_weights,
                      h.lggen_gpu_batch_edges):
                f.restype = i32
            _gpu_handle = h
    return _gpu_handle


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_LIB)
            u64, u32, i32, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
            p = ctypes.POINTER
            h.lggen_rmat.argtypes = [i32, i32, dbl, dbl, dbl, u64, i32, i32, i32, p(_Csr)]
            h.lggen_community.argtypes = [i32, i32, u32, dbl, dbl, dbl, u64, i32, i32, p(_Csr)]
            h.lggen_from_edges.argtypes = [u64, u64, p(u32), p(u32), i32, u64, p(_Csr)]
            h.lggen_sources.argtypes = [u64, p(u64), u32, u64, p(u32)]
            h.lggen_free.argtypes = [p(_Csr)]
            h.lggen_rmat_perm.argtypes = [i32, u64, p(u32)]
            h.lggen_rmat_perm.restype = i32
            h.lggen_hash.argtypes = [u64, u64, u64, u64]
            h.lggen_hash.restype = u64
            for f in (h.lggen_rmat, h.lggen_community, h.lggen_from_edges, h.lggen_sources):
                f.restype = i32
            _handle = h
    return _handle


@dataclass
class Graph:
    """A symmetric CSR graph held in host memory."""

    n: int
    row_ptr: np.ndarray  # uint64[n+1]
    col: np.ndarray  # uint32[arcs]
    weights: Optional[np.ndarray] = None  # uint32[arcs] or None
    name: str = ""

    @property
    def arcs(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


class _Owner:
    """Keeps the C-allocated arrays alive while numpy views exist; frees them after."""

    def __init__(self, c: _Csr):
        self.c = c

    def __del__(self):
        try:
            _lib().lggen_free(ctypes.byref(self.c))
        except Exception:
            pass


def _view(ptr, count, owner):
    a = np.ctypeslib.as_array(ptr, shape=(max(count, 1),))[:count]
    # tie the buffer's lifetime to `owner` through the array's base chain
    holder = np.ndarray(shape=a.shape, dtype=a.dtype, buffer=a)
    holder.flags.writeable = True
    return holder if owner is None else _OwnedArray(holder, owner)


class _OwnedArray(np.ndarray):
    def __new__(cls, arr, owner):
        obj = np.asarray(arr).view(cls)
        obj._owner = owner
        return obj

    def __array_finalize__(self, obj):
        self._owner = getattr(obj, "_owner", None)


def _take(c: _Csr, name: str) -> Graph:
    """Wraps the generator's arrays without copying (large graphs need tens of GB)."""
    n, arcs = int(c.n), int(c.arcs)
    owner = _Owner(c)
    rp = _view(c.row_ptr, n + 1, owner)
    col = _view(c.col, arcs, owner)
    w = _view(c.w, arcs, owner) if bool(c.w) else None
    return Graph(n=n, row_ptr=rp, col=col, weights=w, name=name)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, weighted: bool = False, permute: bool = True, threads: int = 0) -> Graph:
    """R-MAT graph, symmetrized and deduplicated; weights uniform in [1, 255]
    per undirected edge when ``weighted``."""
    out = _Csr()
    _check(_lib().lggen_rmat(scale, edge_factor, a, b, c, seed, int(weighted), int(permute),
                             threads, ctypes.byref(out)), "lggen_rmat")
    return _take(out, f"rmat_s{scale}_ef{edge_factor}_seed{seed}")


def _sort_dedup_rows(rp, deg, col, n: int, chunk: int):
    """Sorts every row of a device CSR and drops duplicate arcs, rows taken in
    chunks of at most ``chunk`` arcs; returns the new (row_ptr, col)."""
    import torch

    dev = col.device
    rp_h = rp.cpu().numpy()
    new_deg = torch.zeros(n, dtype=torch.int64, device=dev)
    w_pos, r0 = 0, 0
    while r0 < n:
        r1 = int(np.searchsorted(rp_h, rp_h[r0] + chunk, side="right")) - 1
        r1 = min(max(r1, r0 + 1), n)
        s0, s1 = int(rp_h[r0]), int(rp_h[r1])
        if s1 > s0:
            rows = torch.repeat_interleave(torch.arange(r1 - r0, device=dev, dtype=torch.int64), deg[r0:r1])
            key = (rows << 32) | (col[s0:s1].to(torch.int64) & 0xFFFFFFFF)
            del rows
            key = torch.sort(key).values
            keep = torch.ones_like(key, dtype=torch.bool)
            keep[1:] = key[1:] != key[:-1]
            key = key[keep]
            del keep
            new_deg[r0:r1] = torch.bincount(key >> 32, minlength=r1 - r0)
            col[w_pos:w_pos + key.numel()] = (key & 0xFFFFFFFF).to(torch.int32)
            w_pos += key.numel()
            del key
        r0 = r1
    col = col[:w_pos].clone()
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(new_deg, 0, out=rp[1:])
    return rp, col


def rmat_gpu(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
             seed: int = 1, weighted: bool = False, permute: bool = True, chunk: int = 1 << 28):
    """The same graph as :func:`rmat`, built on the current CUDA device (for
    scales that take too long on the host).  Returns torch tensors
    ``(row_ptr int64[n+1], col int32[arcs], weights int32[arcs] or None)`` on the
    device holding uint64 / uint32 values; plumbing steps (prefix sums, the
    chunked row sorts, deduplication) use torch."""
    import torch

    lib = _gpu_lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream().cuda_stream
    n, m = 1 << scale, edge_factor << scale
    perm = None
    if permute:
        ph = np.empty(n, dtype=np.uint32)
        _check(_lib().lggen_rmat_perm(scale, seed, ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
               "lggen_rmat_perm")
        perm = torch.from_numpy(ph.view(np.int32)).to(dev)
    pptr = None if perm is None else perm.data_ptr()
    deg = torch.zeros(n, dtype=torch.int64, device=dev)
    _check(lib.lggen_gpu_rmat_count(scale, m, a, a + b, a + b + c, seed, pptr, deg.data_ptr(), st), "rmat_count")
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(deg, 0, out=rp[1:])
    total = int(rp[-1].item())
    col = torch.empty(total, dtype=torch.int32, device=dev)
    cursor = rp[:-1].clone()
    _check(lib.lggen_gpu_rmat_scatter(scale, m, a, a + b, a + b + c, seed, pptr, cursor.data_ptr(),
                                      col.data_ptr(), st), "rmat_scatter")
    del cursor, perm
    rp, col = _sort_dedup_rows(rp, deg, col, n, chunk)
    w = None
    if weighted:
        w = torch.empty(col.numel(), dtype=torch.int32, device=dev)
        _check(lib.lggen_gpu_weights(rp.data_ptr(), col.data_ptr(), n, seed, w.data_ptr(), st), "weights")
    return rp, col, w


def community(log2n: int = 24, log2block: int = 10, zipf_kmax: int = 1 << 14, zipf_s: float = 2.0,
              mean_out: float = 16.0, p_intra: float = 0.9, seed: int = 2, permute: bool = True,
              threads: int = 0) -> Graph:
    """Community-structured graph: Zipf(s) out-degrees scaled to ``mean_out``,
    ``p_intra`` of the out-edges inside the own block, global permutation."""
    out = _Csr()
    _check(_lib().lggen_community(log2n, log2block, zipf_kmax, zipf_s, mean_out, p_intra, seed,
                                  int(permute), threads, ctypes.byref(out)), "lggen_community")
    return _take(out, f"community_n2^{log2n}_b2^{log2block}_seed{seed}")


def from_edges(n: int, edges, weighted: bool = False, seed: int = 0) -> Graph:
    """Symmetric CSR from an explicit undirected edge list (self loops and
    duplicates dropped)."""
    e = np.asarray(edges, dtype=np.uint32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    out = _Csr()
    p32 = ctypes.POINTER(ctypes.c_uint32)
    _check(_lib().lggen_from_edges(n, e.shape[0], src.ctypes.data_as(p32), dst.ctypes.data_as(p32),
                                   int(weighted), seed, ctypes.byref(out)), "lggen_from_edges")
    return _take(out, f"explicit_n{n}")


def sources(g: Graph, count: int, seed: int) -> np.ndarray:
    """``count`` distinct BFS sources drawn uniformly among vertices of nonzero
    degree (Graph500 practice)."""
    out = np.zeros(count, dtype=np.uint32)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    _check(_lib().lggen_sources(g.n, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), count, seed,
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), "lggen_sources")
    return out


def hash4(seed: int, stream: int, i: int, j: int) -> int:
    """The counter-based SplitMix64 draw used by every generator."""
    return int(_lib().lggen_hash(seed, stream, i, j))


@dataclass
class Batch:
    """Independent graphs concatenated: graph g owns vertices
    [vptr[g], vptr[g+1]) and arcs [row_ptr[vptr[g]], row_ptr[vptr[g+1]]);
    col holds LOCAL neighbor IDs (< n_g)."""

    vptr: np.ndarray  # uint64[G+1]
    row_ptr: np.ndarray  # uint64[V+1], global arc offsets
    col: np.ndarray  # uint32[arcs], local IDs
    scales: np.ndarray
    edge_factors: np.ndarray

    @property
    def count(self) -> int:
        return int(self.vptr.shape[0] - 1)

    def graph(self, g: int) -> Graph:
        v0, v1 = int(self.vptr[g]), int(self.vptr[g + 1])
        a0 = int(self.row_ptr[v0])
        rp = (self.row_ptr[v0:v1 + 1] - np.uint64(a0)).astype(np.uint64)
        return Graph(n=v1 - v0, row_ptr=rp, col=self.col[a0:int(self.row_ptr[v1])], name=f"batch[{g}]")


def rmat_batch(count: int = 4096, seed: int = 3, scale_lo: int = 8, scale_hi: int = 16, ef_lo: int = 4,
               ef_hi: int = 32, threads: int = 0) -> Batch:
    """`count` independent R-MAT graphs (a, b, c = .57, .19, .19): graph g has
    scale floor(U), U uniform in [scale_lo, scale_hi + 1) (so n is log-uniform
    over powers of two) and an edge factor uniform in [ef_lo, ef_hi], both
    drawn from SplitMix64(seed, stream 7, g); the graph itself uses seed
    seed * 1000003 + g.  Graphs are built in parallel on the host."""
    from concurrent.futures import ThreadPoolExecutor

    scales, efs = _batch_params(count, seed, scale_lo, scale_hi, ef_lo, ef_hi)
    workers = threads or (os.cpu_count() or 4)

    def one(g):
        return rmat(int(scales[g]), int(efs[g]), seed=seed * 1000003 + g, threads=1)

    with ThreadPoolExecutor(workers) as ex:
        graphs = list(ex.map(one, range(count)))
    ns = np.array([x.n for x in graphs], dtype=np.uint64)
    vptr = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(ns, out=vptr[1:])
    arcs = np.array([x.arcs for x in graphs], dtype=np.uint64)
    abase = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(arcs, out=abase[1:])
    row_ptr = np.empty(int(vptr[-1]) + 1, dtype=np.uint64)
    col = np.empty(int(abase[-1]), dtype=np.uint32)
    for g, x in enumerate(graphs):
        row_ptr[int(vptr[g]):int(vptr[g + 1])] = x.row_ptr[:-1] + abase[g]
        col[int(abase[g]):int(abase[g + 1])] = x.col
    row_ptr[-1] = abase[-1]
    return Batch(vptr=vptr, row_ptr=row_ptr, col=col, scales=scales, edge_factors=efs)


# --- named workloads (synthetic stand-ins for the paper's Kronecker graphs) ---

def rmat_s16_ef16(seed: int = 1) -> Graph:
    """R-MAT scale 16 (65,536 vertices), edge factor 16, unweighted."""
    return rmat(16, 16, seed=seed)


def community_2p24(seed: int = 2, log2n: int = 24) -> Graph:
    """2^24 vertices in 2^14 blocks of 1024, Zipf(2) out-degrees of mean 16,
    90 % intra-block edges, random global permutation."""
    return community(log2n=log2n, log2block=10, seed=seed)


def rmat_s27_ef16_weighted(seed: int = 5, scale: int = 27) -> Graph:
    """R-MAT scale 27, edge factor 16, uniform integer weights in [1, 255]."""
    return rmat(scale, 16, seed=seed, weighted=True)


def _batch_params(count: int, seed: int, scale_lo: int, scale_hi: int, ef_lo: int, ef_hi: int):
    span = scale_hi - scale_lo + 1
    scales = np.array([scale_lo + int((hash4(seed, 7, g, 0) >> 11) * span // (1 << 53)) for g in range(count)])
    efs = np.array([ef_lo + int(hash4(seed, 7, g, 1) % (ef_hi - ef_lo + 1)) for g in range(count)])
    return scales, efs


@dataclass
class DeviceBatch:
    """A batch built on the device: torch tensors vptr int64[G+1], row_ptr
    int64[V+1] (global arc offsets), col int32[arcs] (local IDs)."""

    vptr: object
    row_ptr: object
    col: object
    scales: np.ndarray
    edge_factors: np.ndarray

    @property
    def count(self) -> int:
        return int(self.scales.shape[0])


def rmat_batch_gpu(count: int = 4096, seed: int = 3, scale_lo: int = 8, scale_hi: int = 16, ef_lo: int = 4,
                   ef_hi: int = 32, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                   chunk: int = 1 << 28) -> DeviceBatch:
    """The same batch as :func:`rmat_batch`, built on the current CUDA device:
    every edge of every graph is drawn by one kernel (graph g with its own
    seed seed * 1000003 + g, scale and label table), then rows are sorted and
    deduplicated in chunks."""
    import torch

    lib = _gpu_lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream().cuda_stream
    scales, efs = _batch_params(count, seed, scale_lo, scale_hi, ef_lo, ef_hi)
    ns = (np.ones(count, dtype=np.uint64) << scales.astype(np.uint64))
    ms = efs.astype(np.uint64) * ns
    vptr = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(ns, out=vptr[1:])
    ebase = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(ms, out=ebase[1:])
    seeds = np.array([seed * 1000003 + g for g in range(count)], dtype=np.uint64)
    perms = np.empty(int(vptr[-1]), dtype=np.uint32)
    p32 = ctypes.POINTER(ctypes.c_uint32)
    for g in range(count):
        view = perms[int(vptr[g]):int(vptr[g + 1])]
        _check(_lib().lggen_rmat_perm(int(scales[g]), int(seeds[g]), view.ctypes.data_as(p32)), "lggen_rmat_perm")

    def up(x, dt):
        return torch.from_numpy(np.ascontiguousarray(x).view(dt)).to(dev)

    d_ebase, d_vbase, d_seeds = up(ebase, np.int64), up(vptr[:-1], np.int64), up(seeds, np.int64)
    d_scales, d_perm = up(scales.astype(np.int32), np.int32), up(perms, np.int32)
    V = int(vptr[-1])
    deg = torch.zeros(V, dtype=torch.int64, device=dev)
    args = (d_ebase.data_ptr(), d_vbase.data_ptr(), d_seeds.data_ptr(), d_scales.data_ptr(),
            d_vbase.data_ptr(), d_perm.data_ptr(), count, a, a + b, a + b + c)
    _check(lib.lggen_gpu_batch_edges(0, *args, deg.data_ptr(), None, st), "batch_edges(count)")
    rp = torch.zeros(V + 1, dtype=torch.int64, device=dev)
    torch.cumsum(deg, 0, out=rp[1:])
    col = torch.empty(int(rp[-1].item()), dtype=torch.int32, device=dev)
    cursor = rp[:-1].clone()
    _check(lib.lggen_gpu_batch_edges(1, *args, cursor.data_ptr(), col.data_ptr(), st), "batch_edges(scatter)")
    del cursor, d_perm
    rp, col = _sort_dedup_rows(rp, deg, col, V, chunk)
    return DeviceBatch(vptr=up(vptr, np.int64), row_ptr=rp, col=col, scales=scales, edge_factors=efs)


# --- serving traces ---------------------------------------------------------

@dataclass
class Trace:
    """A request trace for the serving engine, as columns: request i has kind
    (0 lookup, 1 BFS, 2 personalized PageRank), graph, source, lookup vertices
    nbr_vertices[nbr_off[i]:nbr_off[i+1]] and arrival time arrival_ns[i]."""

    kind: np.ndarray
    graph: np.ndarray
    source: np.ndarray
    nbr_off: np.ndarray
    nbr_vertices: np.ndarray
    arrival_ns: np.ndarray

    def __len__(self) -> int:
        return int(self.kind.shape[0])

    def at_rate(self, rate_per_s: float, seed: int = 0) -> "Trace":
        """The same requests with Poisson arrivals at `rate_per_s` (0: all at once)."""
        if rate_per_s <= 0:
            arr = np.zeros(len(self), dtype=np.uint64)
        else:
            rng = np.random.default_rng(seed + 1)
            gaps = rng.exponential(1e9 / rate_per_s, size=len(self))
            arr = np.cumsum(gaps).astype(np.uint64)
        return Trace(self.kind, self.graph, self.source, self.nbr_off, self.nbr_vertices, arr)


def serve_trace(row_ptrs, count: int, seed: int = 4, p_nbr: float = 0.6, p_bfs: float = 0.3,
                max_lookup: int = 256) -> Trace:
    """`count` requests over the graphs whose host row_ptr arrays are given:
    kind drawn with probabilities (p_nbr, p_bfs, rest), graph uniform, lookups
    of 1..max_lookup vertices uniform in [0, n), BFS / PageRank sources uniform
    among vertices of nonzero degree.  Arrivals all at 0 (see Trace.at_rate)."""
    rng = np.random.default_rng(seed)
    u = rng.random(count)
    kind = np.where(u < p_nbr, 0, np.where(u < p_nbr + p_bfs, 1, 2)).astype(np.uint32)
    graph = rng.integers(0, len(row_ptrs), size=count).astype(np.uint32)
    nonzero = [np.flatnonzero(np.diff(np.asarray(rp, dtype=np.uint64)) > 0).astype(np.uint32) for rp in row_ptrs]
    ns = [len(rp) - 1 for rp in row_ptrs]
    source = np.zeros(count, dtype=np.uint32)
    sizes = np.where(kind == 0, rng.integers(1, max_lookup + 1, size=count), 0).astype(np.uint64)
    nbr_off = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(sizes, out=nbr_off[1:])
    nbr_vertices = np.zeros(int(nbr_off[-1]), dtype=np.uint32)
    for i in range(count):
        g = int(graph[i])
        if kind[i] == 0:
            nbr_vertices[int(nbr_off[i]):int(nbr_off[i + 1])] = rng.integers(0, ns[g], size=int(sizes[i]))
        else:
            source[i] = nonzero[g][rng.integers(0, len(nonzero[g]))]
    return Trace(kind, graph, source, nbr_off, nbr_vertices, np.zeros(count, dtype=np.uint64))
