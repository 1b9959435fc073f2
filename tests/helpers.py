"""Small pure-Python helpers for building test inputs (no method arithmetic)."""
import itertools

import numpy as np


def csr_from_edges(n, edges, weights=None):
    """Symmetric CSR (sorted rows) from undirected edges; weights per edge."""
    adj = [dict() for _ in range(n)]
    for k, (u, v) in enumerate(edges):
        if u == v:
            continue
        w = 0 if weights is None else weights[k]
        adj[u][v] = w
        adj[v][u] = w
    rp = [0]
    col, wt = [], []
    for u in range(n):
        for v in sorted(adj[u]):
            col.append(v)
            wt.append(adj[u][v])
        rp.append(len(col))
    return (np.array(rp, dtype=np.uint64), np.array(col, dtype=np.uint32),
            None if weights is None else np.array(wt, dtype=np.uint32))


def all_graphs(n):
    """Every simple undirected graph on n labelled vertices."""
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


def parse_golden(path):
    """Parse a golden fixture: {section: {key: int | [ints] | str}}."""
    out, cur = {}, None
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        if line.startswith("["):
            cur = line.strip("[]").strip()
            out[cur] = {}
            continue
        k, v = (t.strip() for t in line.split("=", 1))
        if k == "edges":
            out[cur][k] = [tuple(int(x) for x in e.split("-")) for e in v.split(",")]
        elif "," in v:
            out[cur][k] = [int(x, 0) for x in v.split(",")]
        else:
            out[cur][k] = int(v, 0)
    return out


def ceil_log2(x):
    """Smallest k with 2^k >= x (x >= 1): the paper's ceil(log x)."""
    k = 0
    while (1 << k) < x:
        k += 1
    return k


def words_to_int(words, nbits):
    """The first nbits of a little-endian u64 word array as a Python int."""
    v = 0
    for i, w in enumerate(words):
        v |= int(w) << (64 * i)
    return v & ((1 << nbits) - 1) if nbits else 0
