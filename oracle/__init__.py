"""CPU oracle for the Log(Graph) hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (the CUDA library and its binding) never imports it, and the two share no
code: the oracle is plain C (``lg_oracle.c``) that sets and reads one bit at a
time, written from the paper's definitions (Sections 3.2-3.7, 4.1-4.3, 5.6 and
7.1.2 of arXiv:2010.15879; see the header of ``lg_oracle.c`` for the readings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "lg_oracle.c")
_LIB = os.path.join(_DIR, "liblgoracle.so")
_lock = threading.Lock()
_handle = None

ID_GLOBAL, ID_LOCAL, ID_LOCAL_GAP = 0, 1, 2
RELABEL_NONE, RELABEL_DM, RELABEL_GREEDY = 0, 1, 2
OFF_PACKED, OFF_EF = 0, 1

_u64, _u32, _i32, _i64, _dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_p = ctypes.POINTER


class _Info(ctypes.Structure):
    _fields_ = [
        ("n", _u64), ("arcs", _u64),
        ("id_mode", _u32), ("off_mode", _u32), ("relabel", _u32), ("sample", _u32), ("weighted", _u32),
        ("s", _u32), ("H", _u32), ("omega", _u32), ("r", _u32), ("w_O", _u32), ("ef_l", _u32),
        ("bits_A", _u64), ("bits_O", _u64), ("ef_N", _u64), ("ef_U", _u64), ("ef_low_bits", _u64),
        ("ef_high_bits", _u64), ("n_samples", _u64),
        ("words_A", _u64), ("words_O", _u64), ("words_ef_low", _u64), ("words_ef_high", _u64),
        ("words_samples", _u64),
        ("A", _p(_u64)), ("O", _p(_u64)), ("ef_low", _p(_u64)), ("ef_high", _p(_u64)),
        ("samples", _p(_u64)), ("x", _p(_u64)),
        ("perm", _p(_u32)), ("inv_perm", _p(_u32)),
    ]


def build(force: bool = False) -> str:
    """Compile ``liblgoracle.so`` next to its source (plain C, -O2, no SIMD flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_LIB)
            h.orc_bits.argtypes = [_u64]
            h.orc_bits.restype = _u32
            h.orc_encode.argtypes = [_u64, _u64, _p(_u64), _p(_u32), _p(_u32), _u32, _u32, _u32, _u32, _u32,
                                     _p(ctypes.c_void_p)]
            h.orc_encode.restype = _i32
            h.orc_free.argtypes = [ctypes.c_void_p]
            h.orc_get_info.argtypes = [ctypes.c_void_p, _p(_Info)]
            for f in ("orc_ef_select", "orc_ef_select_linear", "orc_offset", "orc_degree"):
                getattr(h, f).argtypes = [ctypes.c_void_p, _u64]
                getattr(h, f).restype = _u64
            for f in ("orc_decode_raw", "orc_neighbors"):
                getattr(h, f).argtypes = [ctypes.c_void_p, _u64, _p(_u32), _p(_u32), _u64]
                getattr(h, f).restype = _u64
            h.orc_bfs.argtypes = [_u64, _p(_u64), _p(_u32), _u32, _p(_u32)]
            h.orc_bfs.restype = _i32
            h.orc_sssp.argtypes = [_u64, _p(_u64), _p(_u32), _p(_u32), _u32, _p(_u64)]
            h.orc_sssp.restype = _i32
            h.orc_pagerank.argtypes = [_u64, _p(_u64), _p(_u32), _dbl, _u32, _i64, _p(_dbl)]
            h.orc_pagerank.restype = _i32
            h.orc_pagerank_threads.argtypes = [_u64, _p(_u64), _p(_u32), _dbl, _u32, _i64, _p(_dbl), _i32]
            h.orc_pagerank_threads.restype = _i32
            h.orc_ef_words.argtypes = [_u64, _u64, _u32, _p(_u64), _p(_u64), _p(_u64), _p(_u32)]
            h.orc_ef_words.restype = None
            h.orc_ef_build.argtypes = [_u64, _p(_u64), _u32, _p(_u64), _p(_u64), _p(_u64)]
            h.orc_ef_build.restype = _i32
            h.orc_global_words.argtypes = [_u64, _p(_u32), _p(_u32), _u32, _u32, _u64, _u64, _p(_u64)]
            h.orc_global_words.restype = _i32
            _handle = h
    return _handle


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(_p(ct))


def bits(x: int) -> int:
    """bits(x): 0 for x = 0, else floor(log2 x) + 1."""
    return int(_lib().orc_bits(int(x)))


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


class Encoded:
    """A graph encoded by the oracle; arrays are host numpy copies."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        info = _Info()
        _lib().orc_get_info(self._h, ctypes.byref(info))
        self.info = {k: getattr(info, k) for k, _ in _Info._fields_ if not k[0].isupper() and k not in
                     ("ef_low", "ef_high", "samples", "x", "perm", "inv_perm")}
        self.info["H"] = info.H
        n = info.n

        def arr(ptr, count, dt):
            if not bool(ptr) or count == 0:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(ptr, shape=(int(count),)).copy().astype(dt, copy=False)

        self.A = arr(info.A, info.words_A, np.uint64)
        self.O = arr(info.O, info.words_O, np.uint64)
        self.ef_low = arr(info.ef_low, info.words_ef_low, np.uint64)
        self.ef_high = arr(info.ef_high, info.words_ef_high, np.uint64)
        self.samples = arr(info.samples, info.words_samples, np.uint64)
        self.x = arr(info.x, n + 1, np.uint64)
        self.perm = arr(info.perm, n if info.relabel else 0, np.uint32)
        self.inv_perm = arr(info.inv_perm, n if info.relabel else 0, np.uint32)

    def __getattr__(self, k):
        info = self.__dict__.get("info")
        if info is not None and k in info:
            return info[k]
        raise AttributeError(k)

    def close(self):
        if self._h is not None and self._h.value:
            _lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ef_select(self, j: int) -> int:
        return int(_lib().orc_ef_select(self._h, j))

    def ef_select_linear(self, j: int) -> int:
        return int(_lib().orc_ef_select_linear(self._h, j))

    def offset(self, v: int) -> int:
        return int(_lib().orc_offset(self._h, v))

    def degree(self, v: int) -> int:
        return int(_lib().orc_degree(self._h, v))

    def _decode(self, fn, v: int, with_weights: bool):
        d = self.degree(self.perm[v] if (fn == "orc_neighbors" and self.relabel) else v)
        ids = np.zeros(max(d, 1), dtype=np.uint32)
        w = np.zeros(max(d, 1), dtype=np.uint32) if with_weights else None
        got = getattr(_lib(), fn)(self._h, v, _ptr(ids, _u32), _ptr(w, _u32), d)
        if got != d:
            raise OracleError(-1, fn)
        return (ids[:d], w[:d]) if with_weights else ids[:d]

    def decode_raw(self, v: int, with_weights: bool = False):
        """N_v of stored vertex ``v`` in stored labels and stored order."""
        return self._decode("orc_decode_raw", v, with_weights)

    def neighbors(self, v: int, with_weights: bool = False):
        """N_v of ORIGINAL vertex ``v`` as original IDs, ascending."""
        return self._decode("orc_neighbors", v, with_weights)


def encode(n, row_ptr, col, weights=None, id_mode=ID_GLOBAL, off_mode=OFF_PACKED, relabel=False,
           sample=512, weight_bits=0) -> Encoded:
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    cl = np.ascontiguousarray(col, dtype=np.uint32)
    wt = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32)
    h = ctypes.c_void_p()
    rc = _lib().orc_encode(n, cl.shape[0], _ptr(rp, _u64), _ptr(cl, _u32), _ptr(wt, _u32), id_mode, off_mode,
                           int(relabel), sample, weight_bits, ctypes.byref(h))
    if rc != 0:
        raise OracleError(rc, "orc_encode")
    return Encoded(h.value)


def bfs(n, row_ptr, col, src: int) -> np.ndarray:
    """Depths (uint32, UINT32_MAX = unreachable) of a FIFO-queue BFS on the input CSR."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    cl = np.ascontiguousarray(col, dtype=np.uint32)
    out = np.zeros(n, dtype=np.uint32)
    rc = _lib().orc_bfs(n, _ptr(rp, _u64), _ptr(cl, _u32), src, _ptr(out, _u32))
    if rc != 0:
        raise OracleError(rc, "orc_bfs")
    return out


def sssp(n, row_ptr, col, weights, src: int) -> np.ndarray:
    """Shortest-path distances (uint64, UINT64_MAX = unreachable) from src on the
    weighted input CSR, by Dijkstra's algorithm."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    cl = np.ascontiguousarray(col, dtype=np.uint32)
    wt = np.ascontiguousarray(weights, dtype=np.uint32)
    out = np.zeros(n, dtype=np.uint64)
    rc = _lib().orc_sssp(n, _ptr(rp, _u64), _ptr(cl, _u32), _ptr(wt, _u32), src, _ptr(out, _u64))
    if rc != 0:
        raise OracleError(rc, "orc_sssp")
    return out


def pagerank(n, row_ptr, col, damping: float = 0.85, iters: int = 20, personalize: int = -1,
             threads: int = 1) -> np.ndarray:
    """FP64 pull PageRank on the input CSR, exactly ``iters`` iterations
    (``threads`` > 1 splits vertices over OpenMP threads; same result)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    cl = np.ascontiguousarray(col, dtype=np.uint32)
    out = np.zeros(n, dtype=np.float64)
    rc = _lib().orc_pagerank_threads(n, _ptr(rp, _u64), _ptr(cl, _u32), damping, iters, personalize,
                                     _ptr(out, _dbl), threads)
    if rc != 0:
        raise OracleError(rc, "orc_pagerank")
    return out


def ef_build(x, sample: int = 512):
    """Elias-Fano arrays (low, high, samples, l) of the offsets x_0..x_{N-1},
    laid out as :func:`encode` lays them out (Section 4.3)."""
    xv = np.ascontiguousarray(x, dtype=np.uint64)
    N = xv.shape[0]
    lw, hw, sw, l = _u64(), _u64(), _u64(), _u32()
    _lib().orc_ef_words(N, int(xv[-1]), sample, ctypes.byref(lw), ctypes.byref(hw), ctypes.byref(sw),
                        ctypes.byref(l))
    low = np.zeros(lw.value, dtype=np.uint64)
    high = np.zeros(hw.value, dtype=np.uint64)
    smp = np.zeros(sw.value, dtype=np.uint64)
    rc = _lib().orc_ef_build(N, _ptr(xv, _u64), sample, _ptr(low, _u64), _ptr(high, _u64), _ptr(smp, _u64))
    if rc != 0:
        raise OracleError(rc, "orc_ef_build")
    return low, high, smp, int(l.value)


def global_words(col, weights, s: int, omega: int, w0: int, w1: int) -> np.ndarray:
    """Words [w0, w1) of the global-ID A stream of (col, weights) at s + omega
    bits per record (Sections 3.2.1 and 3.3)."""
    cl = np.ascontiguousarray(col, dtype=np.uint32)
    wt = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32)
    out = np.zeros(max(w1 - w0, 1), dtype=np.uint64)
    rc = _lib().orc_global_words(cl.shape[0], _ptr(cl, _u32), _ptr(wt, _u32), s, omega, w0, w1, _ptr(out, _u64))
    if rc != 0:
        raise OracleError(rc, "orc_global_words")
    return out[:w1 - w0]
