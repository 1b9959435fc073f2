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
_lock = threading.Lock()
_handle = None


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


def _take(c: _Csr, name: str) -> Graph:
    n, arcs = int(c.n), int(c.arcs)
    rp = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(c.col, shape=(max(arcs, 1),))[:arcs].copy()
    w = None
    if bool(c.w):
        w = np.ctypeslib.as_array(c.w, shape=(max(arcs, 1),))[:arcs].copy()
    _lib().lggen_free(ctypes.byref(c))
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
