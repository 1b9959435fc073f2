#!/usr/bin/env python3
"""Benchmark of the Log(Graph) hot path on GB300.

One step = one pass of the whole hot path over one synthetic graph resident in
HBM: lg_encode (DM relabel, widths, prefix sums, bit packing, Elias-Fano
offsets), lg_bfs from 16 sources (bit-parallel multi-source sweeps with the
decoder fused into frontier expansion) and lg_pagerank (20 pull iterations with
the decoder fused in), then lg_free.  The same kernels on the uncompressed
32-bit CSR (LG_ID_CSR32) run beside it as the baseline arm.

Metric: GTEPS = traversed edges per second, where a BFS from one source counts
(sum of the degrees of the reached vertices) / 2 (Graph500 convention) and a
PageRank iteration counts every stored arc once.  ``value`` is over the full
step (encode included); the JSON also carries kernel-only BFS / PageRank GTEPS,
the CSR-32 arm, bytes per arc, the roofline of the PageRank kernel and the CPU
oracle baseline.

The ``batch`` workload times the batching subsystem instead: 4,096 independent
R-MAT graphs (scales 8..16, edge factors 4..32), one step = one replay of the
captured persistent launch that encodes every graph with its own widths, runs
BFS from each graph's vertex 0 and 10 PageRank iterations.

The ``serve`` workload measures the serving engine: 3 resident compressed
R-MAT graphs (scales 20, 22, 24, edge factor 16, global IDs + Elias-Fano
offsets), 100,000 requests (60 % lookups of 1-256 vertices, 30 % BFS, 10 %
personalized PageRank of 10 iterations): the highest Poisson arrival rate the
engine sustains (bisection over rates; the burst rate is reported beside it),
then p50 / p99 latency with Poisson arrivals at 0.25, 0.5 and 0.9 of it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lg|reference]
                       [--workload rmat27|community|rmat16|batch|serve|sssp]
The default workload is R-MAT scale 27 (4.2e9 weighted arcs, the largest
configuration on one GPU); its line also carries, under detail.community_2p24,
the community graph with local-gap IDs and DM relabeling (the bytes evidence).
Under torchrun (N > 1) every rank runs an independent replica ("replicas only":
one GPU holds the whole graph, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402  (seeded inputs)

WORKLOADS = {
    # name: (description, generator, encode options, BFS sources, PageRank iterations)
    "community": ("community graph: 2^24 vertices in 2^14 blocks of 1024, Zipf(2) out-degrees mean 16, "
                  "90% intra-block, random global permutation; DM relabel + local-gap IDs + Elias-Fano "
                  "offsets (select sample 512)",
                  lambda: gen.community_2p24(seed=2),
                  dict(id_mode=2, off_mode=1, relabel=True, select_sample=512), 16, 20),
    "rmat16": ("R-MAT scale 16, edge factor 16, (a,b,c)=(.57,.19,.19); global 16-bit IDs + packed offsets",
               lambda: gen.rmat_s16_ef16(seed=1),
               dict(id_mode=0, off_mode=0, relabel=False), 64, 20),
    "rmat27": ("R-MAT scale 27, edge factor 16, (a,b,c)=(.57,.19,.19), weights in [1,255] at 8 bits; DM relabel "
               "(degree descending, Section 5.6) + global 27-bit IDs + Elias-Fano offsets",
               None,  # built on the device (gen.rmat_gpu)
               dict(id_mode=0, off_mode=1, relabel=True, weight_bits=8), 16, 20),
    "batch": ("batch of 4,096 independent R-MAT graphs, (a,b,c)=(.57,.19,.19), scale floor(U[8,17)), edge "
              "factor uniform in [4,32], seeded; per-graph global IDs at bits(n-1) + packed offsets at "
              "bits(arcs); encode + BFS from vertex 0 + 10 PageRank iterations in one graph-captured "
              "persistent launch, autotuned lanes per vertex and team tile",
              None, None, 1, 10),
}
BATCH_COUNT, BATCH_SEED = 4096, 3
WORKLOADS["serve"] = ("serving: 3 resident R-MAT graphs (scales 20, 22, 24, edge factor 16, seed 4), global IDs + "
                      "Elias-Fano offsets; requests 60% neighborhood lookups of 1-256 uniform vertices, 30% "
                      "single-source BFS, 10% personalized PageRank (10 iterations, d=0.85), graph uniform, "
                      "sources uniform over vertices of nonzero degree; Poisson arrivals",
                      None, None, 1, 10)
SERVE_SCALES, SERVE_SEED, SERVE_RATES = (20, 22, 24), 4, (0.25, 0.5, 0.9)
WORKLOADS["sssp"] = ("SSSP (delta-stepping, delta 32) from 4 sources on R-MAT scale 27, edge factor 16, weights in "
                     "[1,255] at 8 bits; DM relabel + global 27-bit IDs + Elias-Fano offsets; CSR-32 with 32-bit "
                     "weights in the same order beside it",
                     None, dict(id_mode=0, off_mode=1, relabel=True, weight_bits=8), 4, 0)
SSSP_DELTA = 32


class Workload:
    """The input graph on the device (and on the host, made on demand)."""

    def __init__(self, name, dev, log2n=None, relabel=None):
        import torch

        self.desc, make, self.opts, self.S, self.T = WORKLOADS[name]
        if relabel is not None and self.opts is not None and bool(self.opts.get("relabel")) != relabel:
            self.opts = dict(self.opts, relabel=relabel)
            self.desc = self.desc + ("; DM relabel (Section 5.6)" if relabel else "; no relabel")
        scale = 27
        if log2n is not None:
            if name == "community":
                make = lambda: gen.community_2p24(seed=2, log2n=log2n)  # noqa: E731
            elif name == "rmat27":
                scale = log2n  # a smaller R-MAT of the same recipe (profiling captures)
            else:
                raise SystemExit("--profile-log2n applies to the community and rmat27 workloads")
        t0 = time.time()
        if make is None:
            rp, col, w = gen.rmat_gpu(scale, 16, seed=5, weighted=True)
            self.rp_d, self.col_d, self.w_d = rp, col, w
            self._host = None
            self.name = f"rmat_s{scale}_ef16_seed5"
        else:
            g0 = make()
            self._host = (g0.row_ptr, g0.col, g0.weights if "weight_bits" in self.opts else None)
            self.rp_d = torch.from_numpy(g0.row_ptr.view(np.int64)).to(dev)
            self.col_d = torch.from_numpy(g0.col.view(np.int32)).to(dev)
            self.w_d = None if self._host[2] is None else torch.from_numpy(self._host[2].view(np.int32)).to(dev)
            self.name = g0.name
        self.n = self.rp_d.numel() - 1
        self.arcs = self.col_d.numel()
        self.deg_d = self.rp_d[1:] - self.rp_d[:-1]
        log(f"generated {self.name}: n={self.n} arcs={self.arcs} in {time.time() - t0:.1f}s")

    def host(self):
        """(row_ptr u64, col u32, weights u32 or None) numpy arrays."""
        if self._host is None:
            w = None if self.w_d is None else self.w_d.cpu().numpy().view(np.uint32)
            self._host = (self.rp_d.cpu().numpy().view(np.uint64), self.col_d.cpu().numpy().view(np.uint32), w)
        return self._host

    def sources(self):
        class _G:
            pass
        _G.n, _G.row_ptr = self.n, self.host()[0]
        return gen.sources(_G, self.S, seed=7)

    def csr_gb(self):
        """Bytes of the input CSR (row_ptr, col, weights) in GB."""
        return ((self.n + 1) * 8 + self.arcs * 4 * (1 if self.w_d is None else 2)) / 1e9

    def teps_bfs(self, depths):
        """Graph500 traversed edges summed over the sources (on the device)."""
        total = 0
        for row in depths:
            total += int(self.deg_d[row != -1].sum().item()) // 2
        return total
HBM_FALLBACK_GBS = 6800.0
# One metric for both arms: GTEPS, a BFS from one source counting (sum of the
# degrees of the reached vertices) / 2 (Graph500) and a PageRank iteration every
# stored arc once.  Each line's config / cpu_baseline says what one step ran.
METRIC_LG = "GTEPS (BFS + PageRank traversed edges per second, Graph500 counting; compressed vs 32-bit CSR)"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def kernel_source_hash(workload="community"):
    """Hash of the sources of the kernel the roofline reports (k_pr_pull, or
    k_batch for the batch workload)."""
    files = ("lg_batch.cu",) if workload == "batch" else ("lg_traverse.cuh", "lg_device.cuh")
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2010_15879_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per launch of the reported kernel from the committed ncu
    summary, only if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("source_sha") != kernel_source_hash(workload):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.f = None

    def __enter__(self):
        if self.idx is None:  # sampling off
            return self
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return None
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        mhz = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def combine_replicas(step_ms, e2e_ms, te_step, world, device=None):
    """Whole-job numbers for `world` independent replicas (one graph per GPU, no
    collective on the data path): every rank traverses te_step edges per step,
    the job's step time is the slowest rank's (max over ranks), and the value
    is all ranks' edges over that time.  Needs an initialized process group
    when world > 1."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([step_ms, e2e_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms, e2e_ms = float(t[0]), float(t[1])
    return (step_ms, e2e_ms, world * te_step / (step_ms * 1e-3) / 1e9,
            world * te_step / (e2e_ms * 1e-3) / 1e9)


# --------------------------------------------------------------------- GPU arm
def time_arms(lg, wl, steps, warmup, dev, barrier, rank, with_csr_dm=True, clocks=True):
    """The hot path timed on the device (inputs resident in HBM): the
    compressed graph and, beside it, the same kernels on the 32-bit CSR (and
    on the CSR relabeled by the same DM permuter when the compressed arm
    relabels).  One step = lg_encode + lg_bfs (S sources) + lg_pagerank (T
    iterations) + lg_free."""
    import torch

    opts, S, T = wl.opts, wl.S, wl.T
    src_d = torch.from_numpy(wl.sources().view(np.int32)).to(dev)
    depths = torch.empty((S, wl.n), dtype=torch.int32, device=dev)
    ranks = torch.empty(wl.n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(o, ev=None):
        if ev: ev[0].record(stream)
        g = lg.lg_encode(wl.rp_d, wl.col_d, wl.w_d, **o)
        if ev: ev[1].record(stream)
        lg.lg_bfs(g, src_d, out=depths)
        if ev: ev[2].record(stream)
        lg.lg_pagerank(g, 0.85, T, out=ranks)
        if ev: ev[3].record(stream)
        st = g.stats()
        g.free()
        return st

    def timed(o, label, sample_clocks=False):
        for _ in range(warmup):
            step(o)
        torch.cuda.synchronize(dev)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        l0 = lg.lg_kernel_launches()
        with ClockSampler(dev.index if sample_clocks else None) as clk:
            start.record(stream)
            for k in range(steps):
                st = step(o, evs[k])
            stop.record(stream)
            torch.cuda.synchronize(dev)
        barrier()
        launches = lg.lg_kernel_launches() - l0
        ms = start.elapsed_time(stop)
        enc = [e[0].elapsed_time(e[1]) for e in evs]
        bfs = [e[1].elapsed_time(e[2]) for e in evs]
        pr = [e[2].elapsed_time(e[3]) for e in evs]
        log(f"[rank {rank}] {wl.name} {label}: step {ms / steps:.2f} ms (encode {np.median(enc):.2f}, "
            f"bfs {np.median(bfs):.2f}, pr {np.median(pr):.2f})")
        return dict(ms=ms, enc=enc, bfs=bfs, pr=pr, stats=st, launches=launches, clocks=clk.summary())

    step(opts)  # TEPS accounting from one untimed run
    torch.cuda.synchronize(dev)
    te_bfs = wl.teps_bfs(depths)
    te_pr = wl.arcs * T
    res = timed(opts, "log(graph)", sample_clocks=clocks)
    csr = timed(dict(id_mode=3, relabel=False), "csr32")
    csr_dm = timed(dict(id_mode=3, relabel=True), "csr32 in DM order") if (with_csr_dm and opts.get("relabel")) else None
    del depths, ranks
    return dict(lg=res, csr=csr, csr_dm=csr_dm, te_bfs=te_bfs, te_pr=te_pr, te_step=te_bfs + te_pr)


def time_decode(lg, wl, dev, reps=5):
    """lg_decode of the compressed graph (a streaming kernel: compressed A
    and O in, the 32-bit CSR out), CUDA events on the launching stream."""
    import torch

    stream = torch.cuda.current_stream(dev)
    g = lg.lg_encode(wl.rp_d, wl.col_d, wl.w_d, **wl.opts)
    dec_rp = torch.empty(wl.n + 1, dtype=torch.int64, device=dev)
    dec_col = torch.empty(wl.arcs, dtype=torch.int32, device=dev)
    lib = lg.load()
    ms = []
    for k in range(reps + 1):
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        rc = lib.lg_decode(g.handle, dec_rp.data_ptr(), dec_col.data_ptr(), None, wl.arcs, stream.cuda_stream)
        d1.record(stream)
        torch.cuda.synchronize(dev)
        if rc != 0:
            raise SystemExit(f"lg_decode failed: {lg.lg_last_error()}")
        if k:
            ms.append(d0.elapsed_time(d1))
    st = g.stats()
    g.free()
    del dec_rp, dec_col
    peak, _ = peaks()
    t = float(np.median(ms))
    alg = (st["bits_A"] + st["bits_O"]) // 8 + 8 * (wl.n + 1) + 4 * wl.arcs
    kern = ("k_dec_flat: row offsets from the offsets + records in arc order, one launch" if wl.opts["id_mode"] == 0
            else "k_dec_local: row offsets by look-back + per-warp windows staged in shared memory, one launch")
    return {"kernel": f"lg_decode: whole graph to 32-bit CSR ({kern})", "ms": t, "algorithmic_bytes": alg,
            "achieved_gbs": alg / (t * 1e-3) / 1e9, "frac": alg / (t * 1e-3) / 1e9 / peak, "peak_gbs": peak}


def gather_ceiling(lg, table_len, count, dev, reps=5):
    """Rate (G gathers/s) at which the GPU serves uniformly random 4-byte
    reads from a table of `table_len` floats, with the pull kernels' load and
    L2 policy (lg_probe_gather), CUDA events on the launching stream."""
    import torch

    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(12345)
    idx = torch.randint(0, table_len, (count,), dtype=torch.int32, device=dev, generator=g)
    table = torch.rand(table_len, dtype=torch.float32, device=dev)
    out = torch.empty(min(count, lg.PROBE_THREADS), dtype=torch.float32, device=dev)
    ms = []
    for k in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lg.lg_probe_gather(idx, table, out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if k:
            ms.append(e0.elapsed_time(e1))
    del idx, table, out
    t = float(np.median(ms))
    return {"table_bytes": 4 * table_len, "gathers": count, "ms": t, "g_gathers_per_s": count / (t * 1e-3) / 1e9}


def time_e2e(lg, wl, steps, warmup, dev, barrier):
    """End to end through the public API: every step copies its CSR from
    pinned host memory into the device, runs encode + BFS + PageRank and
    reads the depths and ranks back into pinned host memory.  The steps run
    back to back on the compute stream over two preallocated sets of device
    buffers; a copy stream loads the next step's input into the other set and
    reads the previous step's results back while a step computes (events order
    each copy after the compute that frees or fills its buffer)."""
    import torch

    opts, S, T = wl.opts, wl.S, wl.T
    comp = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(dev)
    src_h = wl.sources()
    rp_hn, col_hn, w_hn = wl.host()
    rp_p = torch.from_numpy(rp_hn.view(np.int64)).pin_memory()
    col_p = torch.from_numpy(col_hn.view(np.int32)).pin_memory()
    w_p = None if w_hn is None else torch.from_numpy(w_hn.view(np.int32)).pin_memory()
    src_p = torch.from_numpy(src_h.view(np.int32)).pin_memory()

    def dev_like(t):
        return None if t is None else torch.empty(t.shape, dtype=t.dtype, device=dev)

    # input set 0 is the workload's own device copy (overwritten with the same bytes)
    ins = [(wl.rp_d, wl.col_d, wl.w_d, dev_like(src_p)),
           (dev_like(rp_p), dev_like(col_p), dev_like(w_p), dev_like(src_p))]
    dep_d = [torch.empty((S, wl.n), dtype=torch.int32, device=dev) for _ in range(2)]
    rk_d = [torch.empty(wl.n, dtype=torch.float32, device=dev) for _ in range(2)]
    dep_p = [torch.empty((S, wl.n), dtype=torch.int32).pin_memory() for _ in range(2)]
    rk_p = [torch.empty(wl.n, dtype=torch.float32).pin_memory() for _ in range(2)]
    ev = lambda: torch.cuda.Event()  # noqa: E731
    in_ready = [ev(), ev()]      # input set i loaded
    comp_done = [ev(), ev()]     # the step on set i finished (its input and outputs free to copy)
    out_copied = [ev(), ev()]    # results of set i read back
    for i in range(2):
        comp_done[i].record(comp)
        out_copied[i].record(comp)

    def load(i):
        rp_i, col_i, w_i, src_i = ins[i]
        copy.wait_event(comp_done[i])
        with torch.cuda.stream(copy):
            rp_i.copy_(rp_p, non_blocking=True)
            col_i.copy_(col_p, non_blocking=True)
            if w_i is not None:
                w_i.copy_(w_p, non_blocking=True)
            src_i.copy_(src_p, non_blocking=True)
        in_ready[i].record(copy)

    def run(k, total):
        """step k: compute on set k & 1, then queue the next load and this read-back"""
        i = k & 1
        rp_i, col_i, w_i, src_i = ins[i]
        comp.wait_event(in_ready[i])
        comp.wait_event(out_copied[i])
        g = lg.lg_encode(rp_i, col_i, w_i, stream=comp, **opts)
        lg.lg_bfs(g, src_i, out=dep_d[i], stream=comp)
        lg.lg_pagerank(g, 0.85, T, out=rk_d[i], stream=comp)
        g.free(stream=comp)
        comp_done[i].record(comp)
        if k + 1 < total:
            load(1 - i)
        copy.wait_event(comp_done[i])
        with torch.cuda.stream(copy):
            dep_p[i].copy_(dep_d[i], non_blocking=True)
            rk_p[i].copy_(rk_d[i], non_blocking=True)
        out_copied[i].record(copy)

    def loop(total):
        load(0)
        for k in range(total):
            run(k, total)

    torch.cuda.synchronize(dev)
    loop(max(2, warmup))
    torch.cuda.synchronize(dev)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = []
    e0.record(comp)
    copy.wait_stream(comp)
    load(0)
    for k in range(steps):
        run(k, steps)
        mk = torch.cuda.Event(enable_timing=True)
        mk.record(copy)
        marks.append(mk)
    comp.wait_stream(copy)
    e1.record(comp)
    torch.cuda.synchronize(dev)
    barrier()
    done = [e0.elapsed_time(m) for m in marks]
    ms = e0.elapsed_time(e1) / steps
    h2d = rp_p.numel() * 8 + col_p.numel() * 4 + (0 if w_p is None else w_p.numel() * 4) + S * 4
    d2h = S * wl.n * 4 + wl.n * 4
    del ins[1], dep_d, rk_d, dep_p, rk_p
    return dict(ms=ms, h2d=h2d, d2h=d2h, done=done)


def arms_detail(wl, arms, dec=None):
    """Kernel-level comparison of one workload: bytes, BFS / PageRank GTEPS,
    compressed against the 32-bit CSR through the same kernels."""
    T = wl.T
    res, csr, csr_dm = arms["lg"], arms["csr"], arms["csr_dm"]
    st = res["stats"]
    steps = len(res["enc"])
    pr_ms = float(np.median(res["pr"])) / T
    bfs_ms = float(np.median(res["bfs"]))
    csr_pr_ms = float(np.median(csr["pr"])) / T
    csr_bfs_ms = float(np.median(csr["bfs"]))
    comp = (st["bits_A"] + st["bits_O"]) / 8
    d = {
        "workload": wl.desc, "n": wl.n, "arcs": wl.arcs, "bfs_sources": wl.S, "pr_iters": T,
        "step_ms": res["ms"] / steps, "value_gteps": arms["te_step"] / (res["ms"] / steps * 1e-3) / 1e9,
        "encode_ms": float(np.median(res["enc"])), "bfs_ms": bfs_ms, "pr_ms_per_iter": pr_ms,
        "bfs_gteps": arms["te_bfs"] / (bfs_ms * 1e-3) / 1e9, "pr_gteps": arms["te_pr"] / (pr_ms * T * 1e-3) / 1e9,
        "bits_per_arc": st["bits_per_arc"], "bits_A": st["bits_A"], "bits_O": st["bits_O"],
        "bytes_total": st["bytes_total"],
        "csr32": {"step_ms": csr["ms"] / steps, "encode_ms": float(np.median(csr["enc"])),
                  "bfs_ms": csr_bfs_ms, "pr_ms_per_iter": csr_pr_ms,
                  "bfs_gteps": arms["te_bfs"] / (csr_bfs_ms * 1e-3) / 1e9,
                  "pr_gteps": arms["te_pr"] / (csr_pr_ms * T * 1e-3) / 1e9,
                  "bytes_payload": 4 * wl.arcs + 8 * (wl.n + 1),
                  "value_gteps": arms["te_step"] / (csr["ms"] / steps * 1e-3) / 1e9},
        "csr32_dm_order": None if csr_dm is None else {
            "note": "the same uncompressed CSR relabeled by the same DM permuter",
            "step_ms": csr_dm["ms"] / steps, "encode_ms": float(np.median(csr_dm["enc"])),
            "bfs_ms": float(np.median(csr_dm["bfs"])), "pr_ms_per_iter": float(np.median(csr_dm["pr"])) / T,
            "bfs_gteps_vs": float(np.median(csr_dm["bfs"])) / bfs_ms,
            "pr_gteps_vs": float(np.median(csr_dm["pr"])) / T / pr_ms,
            "value_gteps": arms["te_step"] / (csr_dm["ms"] / steps * 1e-3) / 1e9},
        "bfs_gteps_vs_csr32": csr_bfs_ms / bfs_ms, "pr_gteps_vs_csr32": csr_pr_ms / pr_ms,
    }
    if wl.w_d is None:
        d["bytes_vs_csr32"] = comp / (4 * wl.arcs + 8 * (wl.n + 1))
    else:
        # weighted: against the weighted CSR (32-bit IDs + 32-bit weights), and the
        # same graph encoded without weights against the unweighted CSR-32
        d["bytes_vs_weighted_csr32"] = comp / (8 * wl.arcs + 8 * (wl.n + 1))
        unw_bits = st["bits_A"] // (st["s"] + st["omega"]) * st["s"] if st["id_mode"] == 0 else None
        d["bytes_unweighted_vs_csr32"] = (None if unw_bits is None else
                                          (unw_bits + st["bits_O"]) / 8 / (4 * wl.arcs + 8 * (wl.n + 1)))
    if dec is not None:
        d["decode"] = dec
    return d


def run_lg(args, rank, world):
    import torch

    import paper_2010_15879_gb300 as lg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lg.load(auto_build=True)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    wl = Workload(args.workload, dev, relabel=args.relabel)
    arms = time_arms(lg, wl, args.steps, args.warmup, dev, barrier, rank)
    dec = time_decode(lg, wl, dev)
    e2e = time_e2e(lg, wl, args.steps, args.warmup, dev, barrier)
    res = arms["lg"]
    st = res["stats"]
    T = wl.T
    pr_ms_iter = float(np.median(res["pr"])) / T
    # algorithmic bytes of one PageRank pull launch: the compressed A and O
    # payload, a 4 B contribution gather per arc and a 4 B contribution write
    # per vertex
    alg_bytes = (st["bits_A"] + st["bits_O"]) // 8 + 4 * wl.arcs + 4 * wl.n
    peak, peak_kind = peaks()
    achieved = alg_bytes / (pr_ms_iter * 1e-3) / 1e9
    step_ms = res["ms"] / args.steps
    out = {
        "metric": METRIC_LG,
        "value": None, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 ids / fp32 ranks", "data": "synthetic (seeded generator; no dataset)",
        "config": {"workload": wl.desc, "n": wl.n, "arcs": wl.arcs, "bfs_sources": wl.S, "pr_iters": T,
                   "damping": 0.85, "step": f"lg_encode + lg_bfs ({wl.S} sources) + lg_pagerank ({T} iterations) "
                   "+ lg_free", "l2": "inputs larger than L2 (CSR %.2f GB)" % wl.csr_gb(),
                   "parallelism": f"replicas x{world}"},
    }
    step_ms, e2e_ms, value, e2e_value = combine_replicas(step_ms, e2e["ms"], arms["te_step"], world, dev)
    out["ms_per_step"] = step_ms
    out["value"] = value
    out["e2e"] = {"value": e2e_value, "unit": "GTEPS", "ms_per_step": e2e_ms,
                  "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                  "overlap": "a copy stream loads step k+1's input and reads step k-1's results back while step "
                             "k computes (two preallocated device buffer sets)", "step_done_ms": e2e["done"]}
    out["gpu_launches"] = int(res["launches"])
    out["detail"] = arms_detail(wl, arms, dec)
    out["roofline"] = {"kernel": "k_pr_pull (PageRank pull iteration, decode fused)", "bound": "hbm",
                       "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "peak_kind": f"{peak_kind} (copy bandwidth)",
                       "algorithmic_bytes_per_launch": alg_bytes,
                       "traffic": ncu_traffic(args.workload)}
    # the rate of scattered 4-byte reads the PageRank gathers run into: at the
    # workload's contribution-array size and at an L2-resident 64 MiB
    cnt = min(wl.arcs, 1 << 30)
    ceil_full = gather_ceiling(lg, wl.n, cnt, dev)
    ceil_l2 = gather_ceiling(lg, 1 << 24, cnt, dev)
    pr_rate = wl.arcs / (pr_ms_iter * 1e-3) / 1e9
    out["detail"]["gather_ceiling"] = {
        "probe": "lg_probe_gather: uniformly random 4-byte gathers + a coalesced index stream",
        "contrib_size": ceil_full, "l2_resident_64MiB": ceil_l2, "pr_gathers_per_s": pr_rate,
        "pr_vs_uniform_at_contrib_size": pr_rate / ceil_full["g_gathers_per_s"],
        "pr_frac_of_l2_resident_ceiling": pr_rate / ceil_l2["g_gathers_per_s"],
        "note": "PageRank gathers one 4-byte contribution per arc; the L2-resident rate is the ceiling when the "
                "gathered rows stay in L2 (DM order keeps the hubs' rows there), the uniform rate at the full array "
                "size is the rate without any locality"}
    out["roofline"]["gather_ceiling_frac"] = pr_rate / ceil_l2["g_gathers_per_s"]
    out["clocks"] = res["clocks"]
    if args.workload == "rmat27" and not args.no_secondary:
        # the local-gap / DM workload beside the headline: the <= 75 % bytes
        # evidence and the local-ID decode
        wl2 = Workload("community", dev)
        arms2 = time_arms(lg, wl2, max(3, args.steps // 4), 3, dev, barrier, rank, clocks=False)
        out["detail"]["community_2p24"] = arms_detail(wl2, arms2, time_decode(lg, wl2, dev))
        del wl2
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rp_hn, col_hn, _ = wl.host()
        out["cpu_baseline"] = cpu_baseline(wl.n, rp_hn, col_hn, wl.sources(), wl.T, args.workload)
    return out, rank


# ------------------------------------------------------------------- batches
def batch_alg_bytes(V, arcs, bits_total, iters):
    """Algorithmic bytes of one batch run: encode reads the CSR and writes the
    streams; BFS decodes every reached neighborhood once, gathers a 4 B depth
    per arc and initialises / queues 4 B per vertex; PageRank reads the
    streams, gathers a 4 B contribution per arc and writes 4 B per vertex per
    iteration, plus the initial contributions and the final ranks."""
    b = bits_total // 8
    encode = 8 * (V + 1) + 4 * arcs + b
    bfs = b + 4 * arcs + 12 * V
    pr = 4 * V + iters * (b + 4 * arcs + 4 * V) + 4 * V
    return encode + bfs + pr


def batch_teps(rp_d, depths):
    """Graph500 traversed edges of the per-graph BFS runs (each graph from its vertex 0)."""
    deg = rp_d[1:] - rp_d[:-1]
    return int(deg[depths != -1].sum().item()) // 2


def run_batch(args, rank, world):
    import torch

    import paper_2010_15879_gb300 as lg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lg.load(auto_build=True)
    desc, _, _, _, T = WORKLOADS["batch"]
    t0 = time.time()
    db = gen.rmat_batch_gpu(count=BATCH_COUNT, seed=BATCH_SEED)
    V, arcs = db.row_ptr.numel() - 1, db.col.numel()
    log(f"generated batch of {BATCH_COUNT}: V={V} arcs={arcs} in {time.time() - t0:.1f}s")
    t0 = time.time()
    b = lg.lg_batch_create(db.vptr, db.row_ptr, db.col, autotune=True)
    info = b.info()
    log(f"created (autotuned) in {time.time() - t0:.1f}s: tile {info['tile_arcs']}, teams {info['teams']} "
        f"(max {info['max_team']}), lanes {info['graphs_by_lanes']}, grid {info['grid']}x{info['threads']}")
    stream = torch.cuda.current_stream(dev)
    depths = torch.empty(V, dtype=torch.int32, device=dev)
    ranks = torch.empty(V, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    lg.lg_batch_run(b, 0.85, T, depths, ranks)
    lg.lg_batch_status(b)
    te_bfs = batch_teps(db.row_ptr, depths)
    te_step = te_bfs + arcs * T
    for _ in range(args.warmup):
        lg.lg_batch_run(b, 0.85, T, depths, ranks)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    l0 = lg.lg_kernel_launches()
    with ClockSampler(dev.index) as clk:
        for e in evs:
            e[0].record(stream)
            lg.lg_batch_run(b, 0.85, T, depths, ranks)
            e[1].record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    launches = lg.lg_kernel_launches() - l0
    lg.lg_batch_status(b)
    per = [e[0].elapsed_time(e[1]) for e in evs]
    step_ms = float(np.sum(per)) / args.steps
    log(f"[rank {rank}] batch: step {step_ms:.2f} ms (min {min(per):.2f}, max {max(per):.2f})")

    # e2e: the CSR from pinned host memory into a batch's input buffers, the
    # run, results back.  A second batch over its own input buffers lets
    # consecutive steps alternate between two batches and two streams, so one
    # step's copies overlap the other's run; every step still copies its CSR
    # in and its depths and ranks out.
    rp_p = db.row_ptr.cpu().pin_memory()
    col_p = db.col.cpu().pin_memory()
    rp2, col2 = db.row_ptr.clone(), db.col.clone()
    b2 = lg.lg_batch_create(db.vptr, rp2, col2, autotune=True)
    e2e_b = [(b, db.row_ptr, db.col), (b2, rp2, col2)]
    e2e_streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    dep_d = [depths, torch.empty_like(depths)]
    rk_d = [ranks, torch.empty_like(ranks)]
    dep_p = [torch.empty(V, dtype=torch.int32).pin_memory() for _ in range(2)]
    rk_p = [torch.empty(V, dtype=torch.float32).pin_memory() for _ in range(2)]
    e2e_k = [0]

    def e2e_step():
        i = e2e_k[0] & 1
        e2e_k[0] += 1
        bb, rp_dev, col_dev = e2e_b[i]
        with torch.cuda.stream(e2e_streams[i]):
            rp_dev.copy_(rp_p, non_blocking=True)
            col_dev.copy_(col_p, non_blocking=True)
            lg.lg_batch_run(bb, 0.85, T, dep_d[i], rk_d[i], stream=e2e_streams[i])
            dep_p[i].copy_(dep_d[i], non_blocking=True)
            rk_p[i].copy_(rk_d[i], non_blocking=True)

    for _ in range(max(2, args.warmup)):
        e2e_step()
    torch.cuda.synchronize(dev)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st_ in e2e_streams:
        st_.wait_stream(stream)
    for _ in range(args.steps):
        e2e_step()
    for st_ in e2e_streams:
        stream.wait_stream(st_)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    lg.lg_batch_status(b)
    lg.lg_batch_status(b2)
    b2.free()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    h2d = (V + 1) * 8 + arcs * 4
    d2h = V * 8

    alg = batch_alg_bytes(V, arcs, info["bits_total"], T)
    peak, peak_kind = peaks()
    achieved = alg / (step_ms * 1e-3) / 1e9
    out = {
        "metric": "GTEPS (batch: per-graph BFS from vertex 0 + 10 PageRank iterations, Log(Graph) encode "
                  "included, one graph launch)",
        "value": None, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 ids / fp32 ranks", "data": "synthetic (seeded generator; no dataset)",
        "config": {"workload": desc, "graphs": BATCH_COUNT, "V": V, "arcs": arcs, "pr_iters": T,
                   "damping": 0.85, "l2": "inputs larger than L2 (CSR %.2f GB)" % ((V + 1) * 8 / 1e9 + arcs * 4 / 1e9),
                   "parallelism": f"replicas x{world}"},
    }
    step_ms, e2e_ms, value, e2e_value = combine_replicas(step_ms, e2e_ms, te_step, world, dev)
    out["ms_per_step"] = step_ms
    out["value"] = value
    out["e2e"] = {"value": e2e_value, "unit": "GTEPS", "ms_per_step": e2e_ms,
                  "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                  "overlap": "two batches on two streams: one step's copies overlap the other's run"}
    out["gpu_launches"] = int(launches)
    out["detail"] = {"bfs_edges": te_bfs, "pr_arcs": arcs * T, "bits_total": info["bits_total"],
                     "bits_per_arc": info["bits_total"] / arcs, "tile_arcs": info["tile_arcs"],
                     "teams": info["teams"], "max_team": info["max_team"], "lanes": info["graphs_by_lanes"],
                     "grid": info["grid"], "threads": info["threads"], "work_items": info["n_items"],
                     "bytes_vs_csr32": (info["bits_total"] / 8) / (4 * arcs + 8 * (V + 1))}
    out["roofline"] = {"kernel": "k_batch (persistent: encode + BFS + PageRank, decode fused)", "bound": "hbm",
                       "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "peak_kind": f"{peak_kind} (copy bandwidth)", "algorithmic_bytes_per_launch": alg,
                       "traffic": ncu_traffic("batch")}
    out["clocks"] = clk.summary()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        vptr = db.vptr.cpu().numpy().view(np.uint64)
        out["cpu_baseline"] = cpu_baseline_batch(vptr, rp_p.numpy().view(np.uint64), col_p.numpy().view(np.uint32),
                                                 T, min_seconds=10.0)
    b.free()
    return out, rank


def latency_summary(lat_ns, kinds):
    ms = lat_ns.astype(np.float64) / 1e6
    out = {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
           "mean_ms": float(ms.mean())}
    for k, name in enumerate(("lookup", "bfs", "ppr")):
        sel = ms[kinds == k]
        if sel.size:
            out[name] = {"p50_ms": float(np.percentile(sel, 50)), "p99_ms": float(np.percentile(sel, 99))}
    return out


def run_serve(args, rank, world):
    """Serving: saturation throughput (burst) and latency at 3 Poisson rates."""
    import torch

    import paper_2010_15879_gb300 as lg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lg.load(auto_build=True)
    desc = WORKLOADS["serve"][0]
    t0 = time.time()
    graphs, rps, sizes = [], [], []
    for sc in SERVE_SCALES:
        rp, col, _ = gen.rmat_gpu(sc, 16, seed=SERVE_SEED)
        g = lg.lg_encode(rp, col, id_mode=0, off_mode=1, relabel=args.serve_relabel)
        st = g.stats()
        graphs.append(g)
        rps.append(rp.cpu().numpy().view(np.uint64))
        sizes.append({"scale": sc, "n": st["n"], "arcs": st["arcs"], "bits_A": st["bits_A"], "bits_O": st["bits_O"]})
        del rp, col
    torch.cuda.empty_cache()
    log(f"3 graphs encoded in {time.time() - t0:.1f}s: " + ", ".join(f"2^{x['scale']}: {x['arcs']} arcs" for x in sizes))
    nreq = args.serve_requests
    tr = gen.serve_trace(rps, nreq, seed=SERVE_SEED)
    h2d = float(np.mean(np.where(tr.kind == 0, np.diff(tr.nbr_off) * 4, 0)) + 32)
    n_of = np.array([x["n"] for x in sizes], dtype=np.float64)
    deg_sum = [np.diff(rp) for rp in rps]
    look = np.zeros(nreq)
    for i in np.flatnonzero(tr.kind == 0):
        vs = tr.nbr_vertices[int(tr.nbr_off[i]):int(tr.nbr_off[i + 1])]
        look[i] = (vs.size + 1) * 8 + 4 * float(deg_sum[int(tr.graph[i])][vs].sum())
    d2h = float(np.mean(np.where(tr.kind == 0, look, 4 * n_of[tr.graph])))
    srv = lg.lg_server_create(graphs, device_bytes=48 << 30, host_bytes=8 << 30)

    def replay(trace, label):
        lat, rs = lg.lg_server_replay(srv, trace.kind, trace.graph, trace.source, trace.nbr_off,
                                      trace.nbr_vertices, trace.arrival_ns)
        thr = len(trace) / (rs["makespan_ns"] * 1e-9)
        log(f"{label}: {len(trace)} requests in {rs['makespan_ns'] / 1e9:.2f}s = {thr:.0f} req/s, "
            f"p50 {np.percentile(lat, 50) / 1e6:.2f} ms, p99 {np.percentile(lat, 99) / 1e6:.2f} ms")
        return lat, rs, thr

    # warm-up: a small burst touches every engine
    warm = gen.serve_trace(rps, 2000, seed=SERVE_SEED + 100)
    replay(warm, "warm-up")
    probe_tr = gen.serve_trace(rps, args.serve_probe_requests, seed=SERVE_SEED + 7)

    def sustained(rate, k):
        """Poisson arrivals at `rate` keep every queue bounded: the server
        completes at the offered rate and the latency of the last fifth of
        the trace is not above that of its second fifth (no growth)."""
        t = probe_tr.at_rate(rate, seed=1000 + k)
        lat, rs, thr = replay(t, f"probe {rate:.0f} req/s")
        q = len(lat) // 5
        early, late = np.median(lat[q:2 * q]), np.median(lat[4 * q:])
        ok = thr >= 0.97 * rate and late <= 1.5 * early + 2e6
        return ok, {"offered_req_per_s": rate, "achieved_req_per_s": thr, "p50_second_fifth_ms": early / 1e6,
                    "p50_last_fifth_ms": late / 1e6, "sustained": bool(ok)}

    l0 = lg.lg_kernel_launches()
    with ClockSampler(dev.index) as clk:
        lat_b, rs_b, burst = replay(tr, "burst")
        # saturation: the highest Poisson rate the server sustains (bisection
        # between 0.25 and 1.0 of the burst throughput on a shorter trace)
        lo, hi, probes = 0.25 * burst, burst, []
        ok, rec = sustained(hi, 0)
        probes.append(rec)
        if ok:
            lo = hi
        else:
            for k in range(1, 7):
                mid = 0.5 * (lo + hi)
                ok, rec = sustained(mid, k)
                probes.append(rec)
                if ok:
                    lo = mid
                else:
                    hi = mid
        sat = lo
        per_rate = {}
        for f in SERVE_RATES:
            rate = f * sat
            lat, rs, thr = replay(tr.at_rate(rate, seed=int(f * 100)), f"rate {f:.2f} x saturation")
            summ = latency_summary(lat, tr.kind)
            q = len(lat) // 5
            summ.update({"offered_req_per_s": rate, "achieved_req_per_s": thr,
                         "p50_second_fifth_ms": float(np.median(lat[q:2 * q]) / 1e6),
                         "p50_last_fifth_ms": float(np.median(lat[4 * q:]) / 1e6)})
            per_rate[str(f)] = summ
    launches = lg.lg_kernel_launches() - l0
    st = lg.lg_server_stats_get(srv)
    times = {}
    for gi, x in enumerate(sizes):
        for k, name in ((1, "bfs_level"), (2, "ppr_sweep"), (0, "lookup_batch")):
            o, ns = lg.lg_server_engine_time(srv, gi, k)
            times[f"2^{x['scale']} {name}"] = {"count": o, "mean_us": ns / 1e3 / max(o, 1)}
    srv.destroy()
    # roofline of the PPR sweep on the 2^24 graph: compressed stream + offsets
    # once, one 32-byte sector of 8 contributions per arc, 32 B written per vertex
    big = sizes[2]
    sweep = times[f"2^{big['scale']} ppr_sweep"]
    alg = (big["bits_A"] + big["bits_O"]) // 8 + 32 * big["arcs"] + 32 * big["n"]
    peak, peak_kind = peaks()
    achieved = alg / (sweep["mean_us"] * 1e-6) / 1e9 if sweep["count"] else None
    for g in graphs:
        g.free()
    out = {
        "metric": "serving throughput at saturation (requests/s; 60% lookups, 30% BFS, 10% PPR over 3 resident "
                  "compressed R-MAT graphs; saturation = the highest Poisson rate with bounded queues), with "
                  "p50/p99 latency at 0.25/0.5/0.9 of it",
        "value": sat * world, "unit": "req/s", "n_gpus": world, "steps": nreq, "warmup": 2000,
        "ms_per_step": 1e3 / sat, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 ids / fp32 ranks", "data": "synthetic (seeded generator and trace; no dataset)",
        "config": {"workload": desc + ("; DM relabel" if args.serve_relabel else "; no relabel"), "graphs": sizes,
                   "requests": nreq, "rates_of_saturation": list(SERVE_RATES),
                   "l2": "graphs larger than L2 (2^24: %.2f GB compressed)" % ((big["bits_A"] + big["bits_O"]) / 8e9),
                   "parallelism": f"replicas x{world}", "step": "one request"},
        "latency": per_rate,
        "e2e": {"value": sat * world, "unit": "req/s", "note": "the serving path is end to end: requests from host "
                "memory, results copied to pinned host memory, timed from scheduled arrival to completion",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "detail": {"burst": {"req_per_s": burst, "p50_ms": float(np.percentile(lat_b, 50) / 1e6),
                             "p99_ms": float(np.percentile(lat_b, 99) / 1e6)},
                   "saturation_search": {"requests_per_probe": args.serve_probe_requests, "probes": probes,
                                         "rule": "completes >= 0.97 x offered and the median latency of the last "
                                                 "fifth <= 1.5 x that of the second fifth + 2 ms"},
                   "server": {k: v for k, v in st.items()}, "engine_device_time": times},
        "roofline": {"kernel": "k_ppr_pull (8 personalized PageRank slots, 2^24 graph; CUDA events on the engine "
                               "stream)", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": None if achieved is None else achieved / peak,
                     "peak_kind": f"{peak_kind} (copy bandwidth)", "algorithmic_bytes_per_launch": alg,
                     "traffic": ncu_traffic("serve")},
        "clocks": clk.summary(),
    }
    return out, rank


def sssp_teps(deg_d, dist):
    """Graph500 counting: (sum of the degrees of the reached vertices) / 2."""
    return int(deg_d[dist != -1].sum().item()) // 2


def run_sssp(args, rank, world):
    import torch

    import paper_2010_15879_gb300 as lg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lg.load(auto_build=True)
    desc, _, opts, S, _ = WORKLOADS["sssp"]
    t0 = time.time()
    rp, col, w = gen.rmat_gpu(27, 16, seed=5, weighted=True)
    n, arcs = rp.numel() - 1, col.numel()
    deg_d = rp[1:] - rp[:-1]
    class _G:
        pass
    _G.n, _G.row_ptr = n, rp.cpu().numpy().view(np.uint64)
    src = gen.sources(_G, S, seed=7)
    log(f"generated rmat_s27_ef16_seed5 weighted: n={n} arcs={arcs} in {time.time() - t0:.1f}s")
    stream = torch.cuda.current_stream(dev)
    arms = {}
    for name, o in (("log(graph)", opts), ("csr32", dict(id_mode=3, relabel=opts.get("relabel", False)))):
        g = lg.lg_encode(rp, col, w, **o)
        st = g.stats()
        dist = torch.empty(n, dtype=torch.int64, device=dev)
        te = 0
        for s_ in src:  # TEPS accounting, untimed
            lg.lg_sssp(g, int(s_), SSSP_DELTA, out=dist)
            te += sssp_teps(deg_d, dist)
        for _ in range(args.warmup):
            lg.lg_sssp(g, int(src[0]), SSSP_DELTA, out=dist)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = lg.lg_kernel_launches()
        with ClockSampler(dev.index) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                for s_ in src:
                    lg.lg_sssp(g, int(s_), SSSP_DELTA, out=dist)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        arms[name] = dict(ms=ms, te=te, stats=st, launches=lg.lg_kernel_launches() - l0, clocks=clk.summary())
        log(f"[rank {rank}] {name}: {S} SSSP in {ms:.1f} ms = {te / (ms * 1e-3) / 1e9:.2f} GTEPS")
        g.free()
    lgarm, csr = arms["log(graph)"], arms["csr32"]
    # e2e: weighted CSR from pinned host memory, encode, the 4 SSSP, distances back
    rp_p, col_p, w_p = rp.cpu().pin_memory(), col.cpu().pin_memory(), w.cpu().pin_memory()
    out_p = torch.empty(S * n, dtype=torch.int64).pin_memory()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rp.copy_(rp_p, non_blocking=True)
    col.copy_(col_p, non_blocking=True)
    w.copy_(w_p, non_blocking=True)
    g = lg.lg_encode(rp, col, w, **opts)
    dist = torch.empty(n, dtype=torch.int64, device=dev)
    for i, s_ in enumerate(src):
        lg.lg_sssp(g, int(s_), SSSP_DELTA, out=dist)
        out_p[i * n:(i + 1) * n].copy_(dist, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1)
    g.free()
    st = lgarm["stats"]
    step_ms, e2e_ms, value, e2e_value = combine_replicas(lgarm["ms"], e2e_ms, lgarm["te"], world, dev)
    alg = S * ((st["bits_A"] + st["bits_O"]) // 8 + 8 * arcs + 8 * n)
    peak, peak_kind = peaks()
    achieved = alg / (step_ms * 1e-3) / 1e9
    out = {
        "metric": "GTEPS (SSSP delta-stepping from 4 sources, Log(Graph) compressed weighted graph, Graph500 counting)",
        "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 distances, 8-bit weights", "data": "synthetic (seeded generator; no dataset)",
        "config": {"workload": desc, "n": n, "arcs": arcs, "sources": S, "delta": SSSP_DELTA,
                   "l2": "inputs larger than L2 (weighted CSR %.1f GB)" % ((n + 1) * 8 / 1e9 + arcs * 8 / 1e9),
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "GTEPS", "ms_per_step": e2e_ms, "note": "includes the encode",
                "h2d_bytes_per_step": (n + 1) * 8 + arcs * 8, "d2h_bytes_per_step": S * n * 8},
        "gpu_launches": int(lgarm["launches"] // max(args.steps, 1)),
        "detail": {"csr32": {"ms": csr["ms"], "gteps": csr["te"] / (csr["ms"] * 1e-3) / 1e9},
                   "speedup_vs_csr32": csr["ms"] / lgarm["ms"], "bits_per_arc": st["bits_per_arc"],
                   "bytes_vs_weighted_csr32": ((st["bits_A"] + st["bits_O"]) / 8) / (8 * arcs + 8 * (n + 1))},
        "roofline": {"kernel": "k_sssp_relax (delta-stepping relaxation, decode fused)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} (copy bandwidth)",
                     "algorithmic_bytes_per_launch": alg, "note": "per step (4 SSSP): stream + offsets once and "
                     "one 8-byte distance per arc and vertex per source", "traffic": None},
        "clocks": lgarm["clocks"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_sssp()
    return out, rank


def cpu_baseline_sssp(scale=22):
    """The oracle's Dijkstra on the same generator at scale 22 (1/32 of the
    graph), one source: a bounded sample of the SSSP workload."""
    import oracle

    h = gen.rmat(scale, 16, seed=5, weighted=True)
    s = int(gen.sources(h, 1, seed=7)[0])
    t0 = time.time()
    d = oracle.sssp(h.n, h.row_ptr, h.col, h.weights, s)
    el = time.time() - t0
    te = int(h.degrees()[d != np.iinfo(np.uint64).max].sum()) // 2
    return {"value": te / el / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"one Dijkstra on R-MAT scale {scale} (same generator, weights, edge factor), {el:.1f} s"}


def cpu_baseline_batch(vptr, rp, col, iters, min_seconds=10.0, max_graphs=None):
    """The oracle as it stands (single-threaded C) on a bounded sample of the
    batch: whole graphs in batch order (BFS from vertex 0 + `iters` PageRank
    iterations each) until about min_seconds."""
    import oracle

    te = 0
    t0 = time.time()
    k = 0
    while k < vptr.shape[0] - 1:
        v0, v1 = int(vptr[k]), int(vptr[k + 1])
        a0, a1 = int(rp[v0]), int(rp[v1])
        grp = (rp[v0:v1 + 1] - np.uint64(a0)).astype(np.uint64)
        gcol = col[a0:a1]
        d = oracle.bfs(v1 - v0, grp, gcol, 0)
        te += int(np.diff(grp).astype(np.int64)[d != 0xFFFFFFFF].sum()) // 2
        oracle.pagerank(v1 - v0, grp, gcol, 0.85, iters)
        te += (a1 - a0) * iters
        k += 1
        el = time.time() - t0
        if el >= min_seconds or (max_graphs and k >= max_graphs):
            break
    el = time.time() - t0
    return {"value": te / el / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"the first {k} graph(s) of the batch (BFS from vertex 0 + {iters} PageRank iterations "
                      f"each), {el:.1f} s"}


# ------------------------------------------------------------------ CPU oracle
def host_cores():
    """Host threads this process may use (os.sched_getaffinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_bfs_teps(n, rp, col, deg, sources, threads):
    """Graph500 edges of oracle BFS runs from `sources`, `threads` of them at
    a time (one BFS per thread; the oracle's BFS is sequential)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    def one(s):
        d = oracle.bfs(n, rp, col, int(s))
        return int(deg[d != 0xFFFFFFFF].sum()) // 2

    if threads == 1:
        return sum(one(s) for s in sources)
    with ThreadPoolExecutor(threads) as ex:
        return sum(ex.map(one, sources))


def cpu_baseline(n, rp, col, src_h, iters, workload):
    """The oracle as it stands (plain C, FP64 PageRank, FIFO BFS) on the box's
    host cores, on bounded samples of the same workload:
      single thread -- BFS from the first source(s), then whole PageRank
                       iterations while the sample is under ~10 s;
      every core    -- one BFS source per thread at once plus whole PageRank
                       iterations split over every core by OpenMP.
    At scale 27 one BFS alone takes ~45 s on one core, so there the single-
    thread sample is one BFS source and the all-core sample is PageRank
    iterations only."""
    import oracle

    cores = host_cores()
    deg = np.diff(rp).astype(np.int64)
    big = col.shape[0] > 1_000_000_000
    # single thread
    t0 = time.time()
    te = oracle_bfs_teps(n, rp, col, deg, src_h[:1], 1)
    nb, npr = 1, 0
    while not big and time.time() - t0 < 10.0:
        oracle.pagerank(n, rp, col, 0.85, 1)
        te += col.shape[0]
        npr += 1
    el1 = time.time() - t0
    single = {"value": te / el1 / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
              "sample": f"{nb} BFS source + {npr} PageRank iteration(s) of the same graph, one thread, {el1:.1f} s"}
    # every core
    t0 = time.time()
    te, nb = 0, 0
    if not big:
        nb = min(cores, len(src_h))
        te += oracle_bfs_teps(n, rp, col, deg, src_h[:nb], cores)
    npr = 0
    while npr < 1 or time.time() - t0 < 10.0:
        oracle.pagerank(n, rp, col, 0.85, 1, threads=cores)
        te += col.shape[0]
        npr += 1
    el = time.time() - t0
    return {"value": te / el / 1e9, "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": (f"{nb} BFS sources on {cores} threads at once + " if nb else "") +
                      f"{npr} PageRank iteration(s) on {cores} OpenMP threads, whole graph, {el:.1f} s "
                      f"(of {iters} in a step)",
            "single_core": single, "host_cores": cores}


def profile_pass(args):
    """One untimed pass of the hot path (encode, BFS, PageRank) for profilers:
    few launches before and after the kernels of interest."""
    import torch

    import paper_2010_15879_gb300 as lg

    lg.load(auto_build=True)
    wl = Workload(args.workload, torch.device("cuda", 0), log2n=args.profile_log2n, relabel=args.relabel)
    opts, T = wl.opts, (args.pr_iters if args.pr_iters is not None else wl.T)
    rp, col, w = wl.rp_d, wl.col_d, wl.w_d
    src = torch.from_numpy(wl.sources().view(np.int32)).cuda()
    if args.profile == "decode":
        g = lg.lg_encode(rp, col, w, **opts)
        for _ in range(3):
            lg.lg_decode(g)
        torch.cuda.synchronize()
        log(f"profile pass decode: {g.stats()['arcs']} arcs")
        g.free()
        return
    if args.profile == "encode":
        g = lg.lg_encode(rp, col, w, **opts)
        torch.cuda.synchronize()
        log(f"profile pass encode: {g.stats()['bits_per_arc']:.2f} bits/arc")
        g.free()
        return
    arms = {"lg": opts, "csr32": dict(id_mode=3, relabel=False)}
    for name in (["lg", "csr32"] if args.profile == "both" else [args.profile]):
        g = lg.lg_encode(rp, col, w, **arms[name])
        lg.lg_bfs(g, src)
        lg.lg_pagerank(g, 0.85, T)
        torch.cuda.synchronize()
        log(f"profile pass {name}: {g.stats()['bits_per_arc']:.2f} bits/arc")
        g.free()


def profile_batch(args):
    """Untimed batch runs for profilers: creation (with autotuning), then two
    replays; pass `-s` to skip the autotuner's launches."""
    import torch

    import paper_2010_15879_gb300 as lg

    lg.load(auto_build=True)
    count = args.batch_count or BATCH_COUNT
    db = gen.rmat_batch_gpu(count=count, seed=BATCH_SEED)
    b = lg.lg_batch_create(db.vptr, db.row_ptr, db.col, autotune=True)
    log(f"profile batch: {b.info()['n_items']} work items, {b.info()['launches']} autotune launches")
    for _ in range(2):
        lg.lg_batch_run(b, 0.85, args.pr_iters if args.pr_iters is not None else 10)
    lg.lg_batch_status(b)
    torch.cuda.synchronize()
    b.free()


def run_reference_serve(args, rank, world):
    """The oracle answering the same request trace on the host cores, one
    request at a time, for a bounded sample (about 2 s per step)."""
    import oracle

    hs = [gen.rmat(sc, 16, seed=SERVE_SEED) for sc in SERVE_SCALES]
    tr = gen.serve_trace([h.row_ptr for h in hs], args.serve_requests, seed=SERVE_SEED)

    def answer(i):
        h = hs[int(tr.graph[i])]
        k = int(tr.kind[i])
        if k == 0:
            vs = tr.nbr_vertices[int(tr.nbr_off[i]):int(tr.nbr_off[i + 1])]
            return [h.col[h.row_ptr[v]:h.row_ptr[v + 1]].copy() for v in vs]
        if k == 1:
            return oracle.bfs(h.n, h.row_ptr, h.col, int(tr.source[i]))
        return oracle.pagerank(h.n, h.row_ptr, h.col, 0.85, 10, personalize=int(tr.source[i]))

    i = 0
    for _ in range(args.warmup):
        answer(i % len(tr)); i += 1
    done, t0 = 0, time.time()
    for _ in range(args.steps):
        ts = time.time()
        while time.time() - ts < 2.0:
            answer(i % len(tr)); i += 1; done += 1
    el = time.time() - t0
    v = done / el
    desc = WORKLOADS["serve"][0]
    return {"impl": "reference", "metric": "serving throughput at saturation (requests/s; 60% lookups, 30% BFS, "
                                           "10% PPR over 3 resident compressed R-MAT graphs), with p50/p99 latency "
                                           "at 0.25/0.5/0.9 of it",
            "value": v, "unit": "req/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 ranks / u32 depths", "data": "synthetic (seeded generator and trace)",
            "config": {"workload": desc, "requests": args.serve_requests, "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": "req/s", "cores": 1, "kind": "oracle",
                             "sample": f"the first {done} requests of the trace, one at a time, {el:.1f} s"},
            "e2e": {"value": v, "unit": "req/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}, rank


def profile_serve(args):
    """Untimed serving pass for profilers: the 2^24 graph of the serve
    workload alone, 16 personalized PageRank requests (two full 8-slot sweeps
    of 10 iterations), then 64 BFS and 64 lookups."""
    import paper_2010_15879_gb300 as lg

    lg.load(auto_build=True)
    rp, col, _ = gen.rmat_gpu(SERVE_SCALES[-1], 16, seed=SERVE_SEED)
    g = lg.lg_encode(rp, col, id_mode=0, off_mode=1, relabel=args.serve_relabel)
    rph = rp.cpu().numpy().view(np.uint64)
    del rp, col
    srv = lg.lg_server_create([g], device_bytes=8 << 30, host_bytes=4 << 30)
    nz = np.flatnonzero(np.diff(rph) > 0)
    rng = np.random.default_rng(SERVE_SEED)
    for kind, count in ((2, 16), (1, 64), (0, 64)):
        for _ in range(count):
            if kind == 0:
                lg.lg_server_submit(srv, 0, 0, vertices=rng.integers(0, len(rph) - 1, 128).astype(np.uint32))
            else:
                lg.lg_server_submit(srv, kind, 0, source=int(nz[rng.integers(0, nz.size)]))
        got = 0
        while got < count:
            got += len(lg.lg_server_wait(srv, 64, 30_000_000))
    ops, ns = lg.lg_server_engine_time(srv, 0, 2)
    log(f"profile serve: {ops} PageRank sweeps, {ns / 1e3 / max(ops, 1):.0f} us each")
    srv.destroy()
    g.free()


def run_reference(args, rank, world):
    import torch

    if args.workload == "serve":
        return run_reference_serve(args, rank, world)
    if args.workload == "sssp":
        desc = WORKLOADS["sssp"][0]
        vals = [cpu_baseline_sssp() for _ in range(max(1, args.steps))]
        v = float(np.mean([x["value"] for x in vals]))
        return {"impl": "reference", "metric": "GTEPS (SSSP delta-stepping from 4 sources, Log(Graph) compressed "
                                               "weighted graph, Graph500 counting)",
                "value": v, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": 0,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u64 distances", "data": "synthetic (seeded generator)",
                "config": {"workload": desc, "parallelism": "host cores"},
                "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": vals[0]["sample"]},
                "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}, rank
    if args.workload == "batch":
        desc, _, _, _, T = WORKLOADS["batch"]
        hb = gen.rmat_batch(count=64, seed=BATCH_SEED)  # the batch's first 64 graphs (seeded per graph)
        for _ in range(args.warmup):
            cpu_baseline_batch(hb.vptr, hb.row_ptr, hb.col, T, min_seconds=0.0, max_graphs=1)
        t0 = time.time()
        vals = [cpu_baseline_batch(hb.vptr, hb.row_ptr, hb.col, T, min_seconds=2.0)["value"]
                for _ in range(args.steps)]
        el = time.time() - t0
        v = float(np.mean(vals))
        sample = f"per step: whole graphs from the start of the batch for about 2 s (BFS + {T} PageRank iterations)"
        return {"impl": "reference", "metric": "GTEPS (batch: per-graph BFS from vertex 0 + 10 PageRank "
                                               "iterations, Log(Graph) encode included, one graph launch)",
                "value": v, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 ranks / u32 depths", "data": "synthetic (seeded generator)",
                "config": {"workload": desc, "graphs": BATCH_COUNT, "pr_iters": T, "parallelism": "host cores"},
                "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}, rank

    dev = torch.device("cuda", 0) if (args.workload == "rmat27" and torch.cuda.is_available()) else None
    if args.workload == "rmat27":
        wl = Workload(args.workload, dev)
        n, (rp, col, _), src_h, desc, S, T = wl.n, wl.host(), wl.sources(), wl.desc, wl.S, wl.T
        del wl
        torch.cuda.empty_cache()
    else:
        desc, make, opts, S, T = WORKLOADS[args.workload]
        g0 = make()
        n, rp, col = g0.n, g0.row_ptr, g0.col
        src_h = gen.sources(g0, S, seed=7)
    import oracle

    cores = host_cores()
    deg = np.diff(rp).astype(np.int64)
    big = col.shape[0] > 1_000_000_000

    def unit(k):
        """One bounded step: on the whole input CSR, one PageRank iteration
        on every core (OpenMP), plus, below 10^9 arcs, BFS from `cores`
        sources at once (one per thread)."""
        te = 0
        if not big:
            srcs = [src_h[(k * cores + i) % len(src_h)] for i in range(cores)]
            te += oracle_bfs_teps(n, rp, col, deg, srcs, cores)
        oracle.pagerank(n, rp, col, 0.85, 1, threads=cores)
        return te + col.shape[0]

    for k in range(args.warmup):
        unit(k)
    t0 = time.time()
    te = sum(unit(args.warmup + k) for k in range(args.steps))
    el = time.time() - t0
    v = te / el / 1e9
    sample = ("per step, on the input CSR (no encode): " + ("" if big else f"BFS from {cores} sources at once, one "
              "per thread, + ") + f"1 PageRank iteration on {cores} OpenMP threads")
    out = {"impl": "reference", "metric": METRIC_LG,
           "value": v, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 ranks / u32 depths", "data": "synthetic (seeded generator)",
           "config": {"workload": desc, "n": n, "arcs": int(col.shape[0]), "bfs_sources": S, "pr_iters": T,
                      "step": sample, "parallelism": f"host cores x{cores}"},
           "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return out, rank


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lg", "reference"], default="lg")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat27",
                    help="default: R-MAT scale 27 (the largest configuration that fits one GPU)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--relabel", type=int, choices=[0, 1], default=None,
                    help="override the workload's DM relabeling (Section 5.6): 1 on, 0 off")
    ap.add_argument("--no-secondary", action="store_true",
                    help="rmat27: skip the community 2^24 (local-gap IDs, DM relabel) section of detail")
    ap.add_argument("--profile", choices=["lg", "csr32", "both", "decode", "encode"], default=None,
                    help="run one untimed pass of the hot path (for ncu) and exit: lg / csr32 / both = encode + "
                         "BFS + PageRank of that arm; decode = encode + 3 x lg_decode; encode = one encode")
    ap.add_argument("--pr-iters", type=int, default=None, help="PageRank iterations in --profile mode")
    ap.add_argument("--profile-log2n", type=int, default=None,
                    help="--profile mode of the community / rmat27 workload on a 2^k-vertex graph (a small capture "
                         "case)")
    ap.add_argument("--batch-count", type=int, default=None, help="graphs in --profile mode of the batch workload")
    ap.add_argument("--serve-requests", type=int, default=100000, help="requests per rate (serve workload)")
    ap.add_argument("--serve-probe-requests", type=int, default=30000,
                    help="requests per probe of the sustainable-rate search (serve workload)")
    ap.add_argument("--serve-no-relabel", dest="serve_relabel", action="store_false",
                    help="serve workload: keep the generator's labels (default: DM relabel, Section 5.6, "
                         "which puts the hubs first for gather locality)")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        out, _ = run_reference(args, rank, world)
        print(json.dumps(out), flush=True)
        return
    if args.profile:
        if args.workload == "batch":
            profile_batch(args)
        elif args.workload == "serve":
            profile_serve(args)
        else:
            profile_pass(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    runner = {"batch": run_batch, "serve": run_serve, "sssp": run_sssp}.get(args.workload, run_lg)
    out, rank = runner(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
