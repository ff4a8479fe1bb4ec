#!/usr/bin/env python3
"""Benchmark of the online k-nn graph build (Debatty et al., KDD'16).

Workload (the d = 128 plain FP32 configuration): an exact initial graph of
100,000 points drawn from a 100-component isotropic Gaussian mixture (means
uniform in [-20, 20]^128, sigma 1), k = 10, then a stream of points from the
same mixture inserted in batches of 1,024 (Algorithm 1 per batch: iGNNS with
a budget of n/speedup similarities, expansion 5, then Update to DEPTH 2).

A step is one insert batch of 1,024 points: store, search, intra-batch merge,
Update.  W untimed steps, then K timed steps, each timed with CUDA events on
the stream the library launches on, the L2 flushed between steps.  The
default K + W = 98 batches insert 100,352 points.  One JSON line on stdout.

    python bench.py [--steps K] [--warmup W] [--speedup S] [--impl reference]

--impl reference times the FP64 CPU oracle on this machine's cores instead.
Under torchrun each rank runs an independent replica (its own stream seed);
the value is the inserts of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "inserts+queries/sec at edge recall≥0.95 vs exact; p50/p99 latency; HBM GB/s"
UNIT = "inserts/s"
RECALL_TARGET = 0.95
FALLBACK_BF16_TFLOPS = 1900.0
FALLBACK_HBM_GBS = 6800.0
SEARCH_PROFILE = os.path.join(ROOT, "profiles", "ignns_search_fp32_d128_n100k_batch1024.md")
SEARCH_SOURCES = ("common.cuh", "search.cuh", "search_fp32.cu")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=95)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--speedup", type=float, default=4.0)
    ap.add_argument("--expansion", type=float, default=5.0)
    ap.add_argument("--depth", type=int, default=2)
    ap.add_argument("--workload", default="plain", choices=("small", "plain", "precision"),
                    help="small: d=16, 1,000 + one at a time; plain: d=128, 100,000 + 1,024-point "
                         "batches (default); precision: d=96, 1,000,000 + 1,024-point batches, k=20")
    ap.add_argument("--storage", default=None, choices=("fp32", "bf16", "fp8"),
                    help="searched copy of the rows (default: fp32; bf16 for precision)")
    ap.add_argument("--rescore-mult", type=int, default=4)
    ap.add_argument("--order", default="none", choices=("none", "kmedoids"),
                    help="store the initial points in the order of their balanced k-medoids "
                         "clusters (Algorithm 4; n/1000 clusters) before building the graph")
    ap.add_argument("--experiment", default=None,
                    choices=("search", "depth", "partitions", "serving", "batching", "tail", "growth",
                             "distributed"),
                    help="instead of the benchmark line: the search sweeps (expansion e; "
                         "iGNNS against GNNS at equal evaluations) or the DEPTH sweep, "
                         "one JSON line per point")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the extra records: the precision record (BF16 / FP8 / FP32 searches at "
                         "1,000,000 x 96), the speedup sweep and the query batches")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return FALLBACK_BF16_TFLOPS, "fallback"


def guarded(name, fn, *args, **kwargs):
    """An auxiliary record of the line: fn's result, or, if it raised, the
    error in its place (reported on stderr too), so that the headline line
    is still printed."""
    try:
        return fn(*args, **kwargs)
    except Exception as e:  # noqa: BLE001 -- any failure of an extra record
        msg = f"{type(e).__name__}: {e}"
        print(f"bench.py: {name} record failed: {msg}", file=sys.stderr, flush=True)
        return {"error": msg}


def exact_build_report(W, n, ms, info):
    """The exact graph of n points (tensor-core screening + FP32 settling):
    its time, how many rows the FP32 pass took, and the tensor-pipe view.
    Algorithmic FLOPs are 2 n^2 d (one multiply-add per pair and dimension);
    the screening executes 3 BF16 MMA passes over the dimension padded to
    64 or 128, the rows padded to 128-row blocks and the columns to
    192-column tiles."""
    d = W.mixture.d
    dpt = 64 if d <= 64 else 128
    rows_pad, cols_pad = -(-n // 128) * 128, -(-n // 192) * 192
    alg = 2.0 * n * n * d
    mma = 3 * 2.0 * rows_pad * cols_pad * dpt
    peak, src = bf16_peak()
    return {"n": n, "d": d, "k": W.k, "ms": ms, "path": info["path"],
            "rows_redone": info["rows_redone"], "wait_errors": info["wait_errors"],
            "algorithmic_tflops": alg / ms / 1e9, "mma_tflops": mma / ms / 1e9,
            "tensor_peak": peak, "peak_source": f"{src} bf16_tflops",
            "mma_frac": mma / ms / 1e9 / peak}


def search_source_hash() -> str:
    """Hash of the search kernel's code (comments and blank space removed, so
    that editing a comment does not disown a capture of the same kernel)."""
    h = hashlib.sha256()
    for name in SEARCH_SOURCES:
        with open(os.path.join(ROOT, "paper_1602_06819_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per search launch from the committed ncu summary, if that
    summary was taken on the current search kernel source."""
    try:
        text = open(SEARCH_PROFILE).read()
    except OSError:
        return None, None
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != search_source_hash():
        return None, None
    return float(m_tr.group(1)), os.path.relpath(SEARCH_PROFILE, ROOT)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in out.splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def aggregate_replicas(dist, local_ms: float, local_units: int, device=None):
    """Whole-job figures of N independent replicas: the slowest rank's time
    and the units all ranks processed (barrier on both sides of the timed
    region is the caller's).  With dist None (one process) they are the
    local ones."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_ms, local_units
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def edge_recall(torch, ids, exact):
    """Directed edges u->v present in both graphs, over n*k (Sec. 8.5's e_c)."""
    hit = 0
    for r0 in range(0, ids.shape[0], 16384):
        a, b = ids[r0:r0 + 16384], exact[r0:r0 + 16384]
        hit += int((a[:, :, None] == b[:, None, :]).any(-1).sum().item())
    return hit


def quality_q(e_c, n, n_a, k):
    e_m = n_a * k + n * k * n_a / (n_a + n)
    e_u = (n + n_a) * k - e_m
    return (e_c - e_u) / e_m


# ---------------------------------------------------------------------------
# the CPU oracle, timed (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

ORACLE_MAX_INIT = 100_000


def oracle_initial_graph(W):
    """Untimed setup of the oracle's timed samples: the oracle's exact graph
    (Sec. 2.1) of the workload's initial points (at most the first 100,000:
    the 1,000,000-point workload's would take hours), built on every host
    core.  The lists are kept in the temp directory, keyed by the points and
    the oracle library, so the other arm of the same run on this machine
    reuses them; returns (graph, build seconds, whether it was reused)."""
    import tempfile

    import numpy as np
    import oracle
    lib = oracle.build()
    n0 = min(W.n_init, ORACLE_MAX_INIT)
    X0 = W.initial()[:n0]
    h = hashlib.sha256(X0.tobytes())
    with open(lib, "rb") as f:
        h.update(f.read())
    path = os.path.join(tempfile.gettempdir(), f"knn_oracle_exact_{W.name}_{h.hexdigest()[:16]}.npz")
    t0 = time.perf_counter()
    reused = False
    try:
        z = np.load(path)
        ids, sims = z["ids"], z["sims"]
        reused = ids.shape == (n0, W.k)
    except Exception:
        pass
    if not reused:
        ids, sims, _ = oracle.exact_knn(X0, W.k)
        tmp = path + f".{os.getpid()}.npz"
        np.savez(tmp, ids=ids, sims=sims)
        os.replace(tmp, path)
    g = oracle.Graph(W.mixture.d, W.k, n0 + min(W.n_insert, 20_000))
    g.X[:n0] = X0
    g.ids[:n0] = ids
    g.sims[:n0] = sims
    g.n = n0
    return g, time.perf_counter() - t0, reused


def oracle_cores() -> int:
    return 1  # Algorithm 1 is sequential: the timed inserts use one thread


def run_cpu_baseline(args, W, n_full_avg):
    """Sequential oracle (Algorithm 1, FP64) on the first points of the
    benchmark's own stream, inserted into the oracle's exact graph of the
    initial points: the same workload at the n the GPU run starts from."""
    g, setup_s, reused = oracle_initial_graph(W)
    Xs = W.stream()
    n_start = g.n
    done, t0 = 0, time.perf_counter()
    while done < 16384 and done + 64 <= g.capacity - n_start and \
            time.perf_counter() - t0 < args.cpu_seconds:
        g.insert_stream(Xs[done:done + 64], args.speedup, args.expansion, args.depth,
                        W.seed_search)
        done += 64
    dt = time.perf_counter() - t0
    rate = done / dt
    return {
        "value": rate, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
        "sample": (f"FP64 oracle, Algorithm 1 one point at a time on 1 thread: the first {done} "
                   f"points of this stream inserted into the oracle's exact graph of the "
                   f"{'' if n_start == W.n_init else 'first '}{n_start:,} initial points "
                   f"(n {n_start:,} to {n_start + done:,}; the GPU's "
                   f"timed batches run at mean n {n_full_avg:,.0f}), speedup {args.speedup:g}, "
                   f"e {args.expansion:g}, DEPTH {args.depth}, in {dt:.1f} s; not scaled.  "
                   f"Untimed setup: the oracle's exact initial graph on {os.cpu_count()} host "
                   f"cores, {setup_s:.0f} s{' (reused from this run)' if reused else ''}"),
    }


def run_reference(args, W):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_full_avg = W.n_init + (args.warmup + args.steps / 2) * W.batch
    g, setup_s, reused = oracle_initial_graph(W)
    Xs = W.stream()
    per_step = 64
    if (args.warmup + args.steps) * per_step > g.capacity - g.n:
        per_step = max(1, (g.capacity - g.n) // (args.warmup + args.steps))
    pos = 0
    for _ in range(args.warmup):
        g.insert_stream(Xs[pos:pos + per_step], args.speedup, args.expansion, args.depth,
                        W.seed_search)
        pos += per_step
    n_start = g.n
    step_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        g.insert_stream(Xs[pos:pos + per_step], args.speedup, args.expansion, args.depth,
                        W.seed_search)
        step_s.append(time.perf_counter() - t0)
        pos += per_step
    total = sum(step_s)
    value = args.steps * per_step / total
    sample = (f"FP64 oracle, Algorithm 1 on 1 thread: each step inserts the next {per_step} points "
              f"of this stream one at a time into the oracle's graph (its exact graph of the "
              f"{'' if g.n - pos == W.n_init else 'first '}{g.n - pos:,} initial points, then "
              f"the inserts so far; n {n_start:,} to {g.n:,}; "
              f"the GPU's timed batches run at mean n {n_full_avg:,.0f}); not scaled.  Untimed "
              f"setup: the exact initial graph on {os.cpu_count()} host cores, {setup_s:.0f} s"
              f"{' (reused from this run)' if reused else ''}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, W),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def pick_workload(args):
    from paper_1602_06819_gb300 import inputs
    W = {"small": inputs.SMALL_D16, "plain": inputs.PLAIN_D128,
         "precision": inputs.PRECISION_D96}[args.workload]
    if args.storage is None:
        args.storage = "bf16" if args.workload == "precision" else "fp32"
    return W


def workload_config(args, W):
    cfg = {"workload": W.name, "n_init": W.n_init, "d": W.mixture.d, "k": W.k,
           "components": W.mixture.components, "batch": W.batch,
           "speedup": args.speedup, "expansion": args.expansion, "depth": args.depth,
           "storage": args.storage, "similarity": "1/(1+L2)",
           "inserts_timed_per_gpu": args.steps * W.batch,
           "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}
    if args.storage != "fp32":
        cfg["rescore"] = f"FP32 re-score of the best {args.rescore_mult}k screening candidates"
    if args.order != "none":
        cfg["order"] = (f"initial points stored by balanced k-medoids cluster "
                        f"({kmedoids_clusters(W.n_init)} clusters, imbalance 1.1, 8 chunks, 1 update)")
    return cfg


def kmedoids_clusters(n):
    return max(1, min(1024, n // 1000))


SEQ_RECALL = os.path.join(ROOT, "tests", "golden", "sequential_recall_d128.txt")


def sequential_oracle_recall(args, W, inserts):
    """Graph quality the sequential build (Algorithm 1, FP64 oracle) reaches
    on this stream after the same number of inserts: a stored value, written
    by tests/golden/make_sequential_recall.py from the oracle alone, for the
    d = 128 workload at its default parameters (speedup 4, e 5, DEPTH 2)."""
    from paper_1602_06819_gb300 import inputs
    if (W is not inputs.PLAIN_D128 or (args.speedup, args.expansion, args.depth) != (4.0, 5.0, 2)
            or args.storage != "fp32" or args.order != "none"):
        return None
    try:
        with open(SEQ_RECALL) as f:
            rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    for r in rows:
        if int(r[0]) == inserts:
            return {"edge_recall": float(r[4]), "inserted_recall": float(r[5]), "Q": float(r[6]),
                    "search_evals_per_insert": float(r[7]),
                    "update_evals_per_insert": float(r[8]),
                    "source": os.path.relpath(SEQ_RECALL, ROOT)}
    return None


def recall_record(recall, recall_new, q, n_final, seq):
    """Edge recall (Sec. 8.5's correct edges over n*k) of the final graph and
    of the inserted points' lists alone, beside the sequential oracle's on
    the same stream (batches are held to it within 0.01)."""
    rec = {"edge_recall": recall, "inserted_recall": recall_new, "target": RECALL_TARGET,
           "target_met": recall >= RECALL_TARGET, "Q": q, "n_final": n_final,
           "oracle_sequential": seq}
    if seq is not None:
        d_all = recall - seq["edge_recall"]
        d_new = recall_new - seq["inserted_recall"]
        rec["delta_vs_oracle"] = {"edge_recall": d_all, "inserted_recall": d_new,
                                  "bound": 0.01,
                                  "within": abs(d_all) <= 0.01 and abs(d_new) <= 0.01}
    return rec


def run_speedup_sweep(knn, torch, cfg, X0, Xs, Wm, K, B, exact, flush):
    """The configuration's search-budget sweep: the same stream and batches
    as the headline at speedup 8, 16 and 32 (n / speedup similarities per
    insert), each on a fresh graph from the same exact initial graph;
    inserts/s over the K timed batches (L2 flushed between them), the edge
    recall of all lists and of the inserted lists against the same exact
    graph, and the similarities per insert."""
    import dataclasses
    n0 = X0.shape[0]
    out = []
    for speedup in (8.0, 16.0, 32.0):
        g = knn.Graph(dataclasses.replace(cfg, speedup=speedup), X0)
        for i in range(Wm):
            g.insert(Xs[i * B:(i + 1) * B])
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        st0 = g.stats()
        for i in range(K):
            flush.fill_(float(i))
            a, b = ev[i]
            a.record()
            g.insert(Xs[(Wm + i) * B:(Wm + i + 1) * B])
            b.record()
        torch.cuda.synchronize()
        st1 = g.stats()
        n = st1["n"]
        online = torch.empty((n, exact.shape[1]), dtype=torch.int64, device="cuda")
        g.edges(online)
        g.close()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        out.append({"speedup": speedup, "inserts_per_s": K * B / (ms / 1e3), "ms_per_step": ms / K,
                    "edge_recall": edge_recall(torch, online, exact) / exact.numel(),
                    "inserted_recall": edge_recall(torch, online[n0:], exact[n0:]) / ((n - n0) * exact.shape[1]),
                    "search_evals_per_insert": (st1["search_evals"] - st0["search_evals"]) / (K * B)})
        del online
    return out


def run_query_record(knn, torch, g, W, Xall):
    """Queries (Sec. 3's search, no update) on the final graph: 1,024-query
    batches of the workload's query stream, 5 timed after 1, and their
    recall@k against exhaustive search of the same nodes."""
    Q = torch.from_numpy(W.queries(1024)).cuda()
    k = W.k
    ids = torch.empty((1024, k), dtype=torch.int64, device="cuda")
    g.query(Q, k, 0, ids)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in ev:
        a.record()
        g.query(Q, k, 0, ids)
        b.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    truth = torch.cdist(Q, Xall).topk(k, largest=False).indices
    hit = int((ids[:, :, None] == truth[:, None, :]).any(-1).sum().item())
    return {"batch": 1024, "queries_per_s": 1024 / (ms / 1e3), "ms_per_batch": ms,
            "recall_at_k": hit / truth.numel(), "graph_n": Xall.shape[0]}


def run_precision_record(knn, torch, np, hbm_peak, peak_src, steps=4, warmup=2):
    """The precision workload (1,000,000 initial points, d = 96, 1,000
    components, k = 20), one graph per searched copy: FP32, BF16 and
    FP8-E4M3 screening with an FP32 re-score of the best 4k candidates.  Per
    form: 4 insert batches of the workload's size (8,192 points) after 2,
    49,152 inserts in all, timed as the main line times them (L2 flushed
    between steps), the search kernel's
    roofline, the edge recall of the inserted points' lists against the
    exact graph, and the similarity error against FP64 (numpy, on sampled
    pairs): of the lists' FP32 similarities, and of the screening copy's
    similarities."""
    from paper_1602_06819_gb300 import inputs
    W = inputs.PRECISION_D96
    n0, B, k, d = W.n_init, W.batch, W.k, W.mixture.d
    X0h = W.initial()
    Xsh = W.mixture.sample((steps + warmup) * B, W.seed_stream)
    X0, Xs = torch.from_numpy(X0h).cuda(), torch.from_numpy(Xsh).cuda()
    n_final = n0 + (steps + warmup) * B
    exact = torch.empty((n_final - n0, k), dtype=torch.int64, device="cuda")
    full = torch.empty((n_final, k), dtype=torch.int64, device="cuda")
    knn.knn_exact_graph(torch.cat([X0, Xs]), k, full)
    exact.copy_(full[n0:])
    del full
    rng = np.random.default_rng(7)
    Xcat = np.vstack([X0h, Xsh])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = []
    for storage in ("fp32", "bf16", "fp8"):
        st = {"fp32": knn.KNN_STORAGE_FP32, "bf16": knn.KNN_STORAGE_BF16,
              "fp8": knn.KNN_STORAGE_FP8_E4M3}[storage]
        cfg = knn.GraphConfig(dim=d, k=k, depth=2, storage=st, speedup=4.0, expansion=W.expansion,
                              rescore_mult=4, max_batch=B, seed=W.seed_search, capacity=n_final)
        g = knn.Graph(cfg, X0)
        g.set_timing(True)
        for i in range(warmup):
            g.insert(Xs[i * B:(i + 1) * B])
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        search_ms = 0.0
        torch.cuda.synchronize()
        st0 = g.stats()
        for i in range(steps):
            flush.fill_(float(i))
            a, b = ev[i]
            a.record()
            g.insert(Xs[(warmup + i) * B:(warmup + i + 1) * B])
            b.record()
            search_ms += g.last_timing()["search"]
        torch.cuda.synchronize()
        st1 = g.stats()
        step_ms = sum(a.elapsed_time(b) for a, b in ev)
        ids = torch.empty((n_final, k), dtype=torch.int64, device="cuda")
        sims = torch.empty((n_final, k), dtype=torch.float32, device="cuda")
        g.edges(ids, sims)
        g.close()
        new_ids = ids[n0:]
        recall_new = edge_recall(torch, new_ids, exact) / exact.numel()
        # similarity error against FP64 on sampled (node, neighbour) pairs
        rows = rng.choice(n_final, 2048, replace=False)
        cols = rng.integers(0, k, 2048)
        ih, sh = ids.cpu().numpy(), sims.cpu().numpy()
        nb = ih[rows, cols]
        xa, xb = Xcat[rows].astype(np.float64), Xcat[nb].astype(np.float64)
        s64 = 1.0 / (1.0 + np.linalg.norm(xa - xb, axis=1))
        list_err = np.abs(sh[rows, cols] - s64) / s64
        # the screening similarity: the stored copy of the neighbour's row
        # against the node's FP32 row, in FP64
        Xf = torch.from_numpy(Xcat[nb])
        if storage == "fp32":
            scr = xb
        elif storage == "bf16":
            scr = Xf.bfloat16().double().numpy()
        else:
            scale = Xf.abs().amax(dim=1, keepdim=True).clamp_min(1e-30) / 448.0
            scr = ((Xf / scale).to(torch.float8_e4m3fn).float() * scale).double().numpy()
        s_scr = 1.0 / (1.0 + np.linalg.norm(xa - scr, axis=1))
        scr_err = np.abs(s_scr - s64) / s64
        del ids, sims, new_ids
        dp = 96
        row_bytes = {"fp32": 4 * dp, "bf16": 2 * dp, "fp8": dp + 4}[storage]
        d_evals = st1["search_evals"] - st0["search_evals"]
        d_adj = st1["adjacency_reads"] - st0["adjacency_reads"]
        alg = (d_evals * row_bytes + d_adj * k * 4 + steps * B * 4 * dp) / steps
        launch_ms = search_ms / steps
        achieved = alg / (launch_ms / 1e3) / 1e9
        out.append({
            "storage": storage, "workload": W.name, "n_init": n0, "d": d, "k": k,
            "inserts_per_s": steps * B / (step_ms / 1e3), "ms_per_step": step_ms / steps,
            "search_ms_per_step": launch_ms,
            "inserted_recall": recall_new,
            "evals_per_insert": d_evals / (steps * B),
            "similarity_rel_err_vs_fp64": {
                "lists_max": float(list_err.max()), "lists_median": float(np.median(list_err)),
                "screening_max": float(scr_err.max()),
                "screening_median": float(np.median(scr_err)), "pairs": 2048},
            "roofline": {"kernel": f"ignns_search_kernel<{storage},{dp}>", "bound": "hbm",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_source": f"{peak_src} hbm_gbs",
                         "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms},
            "steps": steps, "warmup": warmup,
            "l2": "flushed between timed steps (256 MiB write)"})
    del flush, X0, Xs, exact
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# experiments (Sec. 8.2, 8.3): the paper's search and depth studies, on the
# GPU path, against the exhaustive search of the same library
# ---------------------------------------------------------------------------

def _exp_line(**kv):
    print(json.dumps(kv), flush=True)


def run_search_experiment(knn, torch, np):
    """Recall@10 of graph searches against exhaustive search (speedup 1, no
    expansion test: linear search), on the exact 10-nn graph of each set.
    (1) the expansion parameter e at a fixed speedup (the study behind the
    paper's expansion figure: 5,000 synthetic points, speedup 50);
    (2) iGNNS (eager climb + expansion test), GNNS (best-neighbour climb, no
    test) and each improvement alone, at equal evaluations (the iGNNS/GNNS
    comparison: 5,000 synthetic points, e = 5)."""
    from paper_1602_06819_gb300 import inputs
    sets = [
        ("gmm-d3-n5000", inputs.Mixture(d=3, components=10, half_width=10.0, sigma=1.0, seed=41),
         5000, 1000, 50.0, (2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0)),
        ("gmm-d128-n100k", inputs.PLAIN_D128.mixture, 100000, 1024, 16.0,
         (2.0, 4.0, 8.0, 16.0, 32.0, 64.0)),
    ]
    k = 10
    for name, mix, n, nq, s_fixed, speedups in sets:
        X = torch.from_numpy(mix.sample(n, 42)).cuda()
        Q = torch.from_numpy(mix.sample(nq, 43)).cuda()
        cfg = knn.GraphConfig(dim=mix.d, k=k, depth=2, speedup=1.0, expansion=math.inf,
                              max_batch=nq, seed=7, capacity=n)
        g = knn.Graph(cfg, X)
        ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        ctr = np.empty((nq, 8), np.int64)

        def run(speedup, e, climb):
            g.set_search(speedup, e, climb)
            g.query(Q, k, 0, ids)
            g.counters(ctr)
            torch.cuda.synchronize()
            return ids.clone(), float(ctr[:, 0].mean())

        truth, ev_all = run(1.0, math.inf, "eager")

        def recall(got):
            return float((got[:, :, None] == truth[:, None, :]).any(-1).float().mean().item())

        for e in (1.01, 1.2, 1.5, 2.0, 3.0, 5.0, 10.0, 20.0, math.inf):
            got, ev = run(s_fixed, e, "eager")
            _exp_line(experiment="expansion", set=name, n=n, queries=nq, k=k, speedup=s_fixed,
                      expansion=None if math.isinf(e) else e, climb="eager", recall=recall(got),
                      evals_per_query=ev)
        for speedup in speedups:
            for label, e, climb in (("iGNNS", 5.0, "eager"), ("GNNS", math.inf, "best"),
                                    ("eager only", math.inf, "eager"), ("expansion only", 5.0, "best")):
                got, ev = run(speedup, e, climb)
                _exp_line(experiment="ignns_vs_gnns", set=name, n=n, queries=nq, k=k,
                          speedup=speedup, method=label, expansion=None if math.isinf(e) else e,
                          climb=climb, recall=recall(got), evals_per_query=ev)
        g.close()


def run_depth_experiment(knn, torch, np):
    """The online build (Algorithm 1, one point at a time) with DEPTH 1..5:
    edge recall and Q of the final graph against its exact graph, and the
    similarities computed per insert (Sec. 8.3's depth study: 1,000 initial
    synthetic points + 1,000 added at speedup 20; and 8,000 + 16,000 at
    speedup 4)."""
    from paper_1602_06819_gb300 import inputs
    k = 10
    runs = [("gmm-d16-1000+1000", inputs.SMALL_D16.mixture, 1000, 1000, 20.0),
            ("gmm-d16-1000+1000", inputs.SMALL_D16.mixture, 1000, 1000, 4.0),
            ("gmm-d16-8000+16000", inputs.SMALL_D16.mixture, 8000, 16000, 4.0)]
    for name, mix, n0, na, speedup in runs:
        X0 = torch.from_numpy(mix.sample(n0, 1)).cuda()
        Xs = torch.from_numpy(mix.sample(na, 2)).cuda()
        Xall = torch.cat([X0, Xs])
        exact = torch.empty((n0 + na, k), dtype=torch.int64, device="cuda")
        knn.knn_exact_graph(Xall, k, exact)
        for depth in (1, 2, 3, 4, 5):
            cfg = knn.GraphConfig(dim=mix.d, k=k, depth=depth, speedup=speedup, expansion=5.0,
                                  max_batch=1, seed=4, capacity=n0 + na)
            g = knn.Graph(cfg, X0)
            st0 = g.stats()
            t0 = time.perf_counter()
            for i in range(na):
                g.insert(Xs[i:i + 1])
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            st1 = g.stats()
            online = torch.empty((n0 + na, k), dtype=torch.int64, device="cuda")
            g.edges(online)
            g.close()
            e_c = edge_recall(torch, online, exact)
            search = (st1["search_evals"] - st0["search_evals"]) / na
            update = (st1["update_evals"] - st0["update_evals"]) / na
            _exp_line(experiment="depth", set=name, n_init=n0, n_added=na, k=k, speedup=speedup,
                      expansion=5.0, depth=depth, edge_recall=e_c / exact.numel(),
                      Q=quality_q(e_c, n0, na, k), search_evals_per_insert=search,
                      update_evals_per_insert=update, inserts_per_s=na / secs)


def run_distributed_experiment(knn, torch, np):
    """The distributed online build (Algorithm 5) on synthetic R^3 data (a
    10-component Gaussian mixture), one point inserted at a time, k = 10,
    speedup 4, e = 5, DEPTH 2, 8 balanced k-medoids partitions of the
    initial points:
    (1) the interval between medoid recomputes (Sec. 8.5): 4,000 initial
        points + 4,000 added, medoids recomputed at every 10 % of growth or
        never, 10 repetitions; correct edges e_c of the final graph;
    (2) graph quality (Sec. 8.5's experiment): 8,000 + 16,000, e_c and Q
        against the exact graph of the points so far every 4,000 inserts,
        beside Algorithm 1 (one partition) on the same stream."""
    from paper_1602_06819_gb300 import inputs
    k, P, speedup, e = 10, 8, 4.0, 5.0

    def build(X0, Xs, interval, parts, seed, checkpoints=()):
        n0, na = X0.shape[0], Xs.shape[0]
        cfg = knn.GraphConfig(dim=X0.shape[1], k=k, depth=2, speedup=speedup, expansion=e,
                              max_batch=max(parts, 1), seed=seed, capacity=n0 + na)
        g = knn.Graph(cfg, X0)
        labels = torch.empty(n0, dtype=torch.int32, device="cuda")
        medoids = torch.empty(parts, dtype=torch.int64, device="cuda")
        knn.knn_balanced_kmedoids(X0, parts, 1.1, 8, 2, seed, labels, medoids)
        g.set_partitions(labels, medoids, interval)
        marks = []
        t0 = time.perf_counter()
        for i in range(na):
            g.insert_distributed(Xs[i:i + 1])
            if i + 1 in checkpoints:
                n = n0 + i + 1
                online = torch.empty((n, k), dtype=torch.int64, device="cuda")
                g.edges(online)
                exact = torch.empty((n, k), dtype=torch.int64, device="cuda")
                knn.knn_exact_graph(torch.cat([X0, Xs[:i + 1]]), k, exact)
                e_c = edge_recall(torch, online, exact)
                marks.append({"added": i + 1, "e_c": e_c, "edge_recall": e_c / exact.numel(),
                              "Q": quality_q(e_c, n0, i + 1, k)})
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        online = torch.empty((n0 + na, k), dtype=torch.int64, device="cuda")
        g.edges(online)
        rec = g.partitions()
        g.close()
        return online, rec, marks, na / secs

    mix = inputs.Mixture(d=3, components=10, half_width=10.0, sigma=1.0, seed=41)
    # (1) recompute interval
    for interval in (0.1, 0.0):
        ecs, recs = [], []
        for rep in range(10):
            X0 = torch.from_numpy(mix.sample(4000, 100 + rep)).cuda()
            Xs = torch.from_numpy(mix.sample(4000, 200 + rep)).cuda()
            exact = torch.empty((8000, k), dtype=torch.int64, device="cuda")
            knn.knn_exact_graph(torch.cat([X0, Xs]), k, exact)
            online, rec, _, rate = build(X0, Xs, interval, P, 300 + rep)
            ecs.append(edge_recall(torch, online, exact))
            recs.append(rec)
        _exp_line(experiment="distributed", study="medoid_interval", set="gmm-d3-4000+4000", parts=P, k=k,
                  speedup=speedup, expansion=e, interval=interval, repetitions=10,
                  e_c_mean=float(np.mean(ecs)), e_c_std=float(np.std(ecs)), e_c_min=int(min(ecs)),
                  e_c_max=int(max(ecs)), edge_recall_mean=float(np.mean(ecs)) / (8000 * k),
                  recomputes=int(recs[0]), inserts_per_s=rate)
    # (2) graph quality over time, beside Algorithm 1
    X0 = torch.from_numpy(mix.sample(8000, 1)).cuda()
    Xs = torch.from_numpy(mix.sample(16000, 2)).cuda()
    marks_at = (4000, 8000, 12000, 16000)
    for parts in (P, 1):
        _, rec, marks, rate = build(X0, Xs, 0.0, parts, 7, marks_at)
        for mk in marks:
            _exp_line(experiment="distributed", study="quality", set="gmm-d3-8000+16000", parts=parts, k=k,
                      speedup=speedup, expansion=e, **mk, inserts_per_s=rate)


def run_partition_experiment(knn, torch, np):
    """Partitioned search (Algorithm 3) on the default workload's 100,000
    initial points stored in the order of P balanced k-medoids clusters:
    recall@10 against exhaustive search, similarities per query, the time of
    a 1,024-query batch and the latency of single queries, for P = 1 (the
    plain search) .. 32, at the same total budget n / speedup."""
    from paper_1602_06819_gb300 import inputs
    W = inputs.PLAIN_D128
    X = torch.from_numpy(W.initial()).cuda()
    Q = torch.from_numpy(W.mixture.sample(1024, W.seed_query)).cuda()
    n, k, nq = X.shape[0], 10, Q.shape[0]
    for speedup in (4.0, 16.0):
        for P in (1, 2, 4, 8, 16, 32):
            if P == 1:
                Xo, offs = X, torch.tensor([0, n], dtype=torch.int64)
            else:
                perm = torch.empty(n, dtype=torch.int64, device="cuda")
                offs = torch.empty(P + 1, dtype=torch.int64, device="cuda")
                knn.knn_balanced_kmedoids(X, P, 1.05, 1, 2, 5, order=perm, offsets=offs)
                Xo = X[perm].contiguous()
                offs = offs.cpu()
            cfg = knn.GraphConfig(dim=W.mixture.d, k=k, depth=2, speedup=1.0, expansion=math.inf,
                                  max_batch=nq, seed=7, capacity=n)
            g = knn.Graph(cfg, Xo)
            ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
            g.query(Q, k, 0, ids)
            truth = ids.clone()
            g.set_search(speedup, 5.0, "eager")
            ctr = np.empty((nq, 8), np.int64)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g.query_partitioned(Q, k, 0, offs, ids)          # warm
            torch.cuda.synchronize()
            e0.record()
            g.query_partitioned(Q, k, 0, offs, ids)
            e1.record()
            torch.cuda.synchronize()
            batch_ms = e0.elapsed_time(e1)
            g.counters(ctr)
            recall = float((ids[:, :, None] == truth[:, None, :]).any(-1).float().mean().item())
            one = torch.empty((1, k), dtype=torch.int64, device="cuda")
            lat = []
            for i in range(64):
                e0.record()
                g.query_partitioned(Q[i:i + 1], k, 10_000 + i, offs, one)
                e1.record()
                torch.cuda.synchronize()
                lat.append(e0.elapsed_time(e1))
            g.close()
            lat.sort()
            _exp_line(experiment="partitions", set="gmm-d128-n100k", n=n, queries=nq, k=k,
                      speedup=speedup, expansion=5.0, parts=P, recall=recall,
                      evals_per_query=float(ctr[:, 0].mean()), batch_ms=batch_ms,
                      single_query_ms_p50=lat[len(lat) // 2], single_query_ms_p99=lat[-1])


def run_serving_experiment(knn, torch, np):
    """The serving pattern: Poisson arrivals of requests (insert : query =
    1 : 4, 1..512 points each, uniform) into the continuous-batching server
    over one growing graph (1,000,000 initial points, d = 128, k = 10,
    BF16 screening with FP32 re-score, speedup 4, e = 5); for each arrival
    rate lambda, about 15 s of traffic: completed points/s, p50/p99 request
    latency (submission to results on the host) and the mean step.  The same
    sweep on the plain FP32 path for comparison; recall@10 of 256 queries
    against exhaustive search on the final graph of each run.  The graph is
    created at its initial size and grows as inserts arrive (admission by
    free device memory: knn_graph_reserve with 8 GiB kept free)."""
    from paper_1602_06819_gb300 import inputs
    import threading
    mix = inputs.Mixture(d=128, components=1000, half_width=20.0, sigma=1.0, seed=51)
    n0, k, seconds = 1_000_000, 10, 15.0
    pool = mix.sample(600_000, 52)
    Qr = mix.sample(256, 53)
    rng = np.random.default_rng(54)
    for storage, lams, parts in (("bf16", (10, 20, 30, 40, 60, 80), 0), ("fp32", (10, 20, 30, 40), 0),
                                 ("bf16", (10, 20, 30), 32)):
        st = {"fp32": knn.KNN_STORAGE_FP32, "bf16": knn.KNN_STORAGE_BF16}[storage]
        cfg = knn.GraphConfig(dim=128, k=k, depth=2, storage=st, speedup=4.0, expansion=5.0,
                              rescore_mult=4, max_batch=1024, seed=9, capacity=n0)
        X0 = torch.from_numpy(mix.sample(n0, 50)).cuda()
        offs = None
        if parts:
            # queries run the partitioned search (Algorithm 3) over the balanced
            # k-medoids clusters of the initial points, stored cluster by cluster
            perm = torch.empty(n0, dtype=torch.int64, device="cuda")
            offs_d = torch.empty(parts + 1, dtype=torch.int64, device="cuda")
            knn.knn_balanced_kmedoids(X0, parts, 1.05, 1, 2, 5, order=perm, offsets=offs_d)
            X0 = X0[perm].contiguous()
            offs = offs_d.cpu().numpy()
        g = knn.Graph(cfg, X0)
        del X0
        used = 0
        for lam in lams:
            o = None
            if parts:   # the parts of the graph as it stands (the last one takes the inserts)
                o = offs.copy()
                o[-1] = g.stats()["n"]
            srv = knn.Server(g, k, 1024, grow_headroom_bytes=8 << 30, part_offsets=o)
            pending = []
            lock = threading.Lock()
            done_evt = threading.Event()
            lat, sizes = [], []

            def waiter():
                while True:
                    with lock:
                        item = pending.pop(0) if pending else None
                    if item is None:
                        if done_evt.is_set():
                            return
                        time.sleep(0.0005)
                        continue
                    rid, m, kind = item
                    _, _, info = srv.wait(rid, m, kind)
                    lat.append(info["latency_ms"])
                    sizes.append(m)

            th = threading.Thread(target=waiter)
            th.start()
            t_start = time.perf_counter()
            t_next = t_start
            nsub = 0
            while t_next - t_start < seconds:
                now = time.perf_counter()
                if now < t_next:
                    time.sleep(min(t_next - now, 0.002))
                    continue
                m = int(rng.integers(1, 513))
                kind = knn.KNN_REQ_INSERT if rng.random() < 0.2 else knn.KNN_REQ_QUERY
                if used + m > pool.shape[0]:
                    used = 0
                vecs = pool[used:used + m]
                used += m
                rid = srv.submit(kind, vecs)
                with lock:
                    pending.append((rid, m, kind))
                nsub += 1
                t_next += rng.exponential(1.0 / lam)
            done_evt.set()
            th.join()
            wall = time.perf_counter() - t_start
            stats = srv.stats()
            srv.close()
            lat.sort()
            _exp_line(experiment="serving", storage=storage, query_parts=parts, lam_requests_per_s=lam, requests=nsub,
                      points_per_s=sum(sizes) / wall, offered_points_per_s=lam * 256.5,
                      p50_ms=lat[len(lat) // 2], p99_ms=lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                      steps=stats["steps"], mean_step_points=stats["points"] / max(1, stats["steps"]),
                      gpu_busy_frac=stats["busy_ms"] / (wall * 1e3), graph_n=g.stats()["n"],
                      graph_capacity=stats["capacity"], grows=stats["grows"],
                      max_queue=stats["max_queue"], seconds=wall)
        # recall@10 of queries on the final graph against exhaustive search
        Q = torch.from_numpy(Qr).cuda()
        ids = torch.empty((256, k), dtype=torch.int64, device="cuda")
        if parts:
            fo = offs.copy()
            fo[-1] = g.stats()["n"]
            g.query_partitioned(Q, k, 0, torch.from_numpy(fo), ids)
        else:
            g.query(Q, k, 0, ids)
        got = ids.clone()
        g.set_search(1.0, math.inf, "eager")
        g.query(Q, k, 0, ids)
        torch.cuda.synchronize()
        rec = float((got[:, :, None] == ids[:, None, :]).any(-1).float().mean().item())
        _exp_line(experiment="serving_recall", storage=storage, query_parts=parts, graph_n=g.stats()["n"],
                  recall_at_10=rec)
        g.close()


def run_growth_experiment(knn, torch, np):
    """The serving pattern's growth: one graph of 1,000,000 points (d = 128,
    1,000 components, k = 10, BF16 screening with FP32 re-score, speedup 4,
    e = 5) created at exactly that size and grown to 5,000,000 through the
    continuous-batching server, which admits inserts by free device memory
    (knn_graph_reserve whenever an insert does not fit, keeping 8 GiB free).
    Insert requests of 512 points are submitted as fast as the server takes
    them, with a 1-point query request every 20th request; every 200,000
    nodes a line reports the graph's size and capacity, the growth steps so
    far, the insert rate of that stretch and the latency of its queries."""
    from paper_1602_06819_gb300 import inputs
    mix = inputs.Mixture(d=128, components=1000, half_width=20.0, sigma=1.0, seed=51)
    n0, n_end, k, req = 1_000_000, 5_000_000, 10, 512
    cfg = knn.GraphConfig(dim=128, k=k, depth=2, storage=knn.KNN_STORAGE_BF16, speedup=4.0,
                          expansion=5.0, rescore_mult=4, max_batch=1024, seed=9, capacity=n0)
    g = knn.Graph(cfg, torch.from_numpy(mix.sample(n0, 50)).cuda())
    pool = mix.sample(400_000, 55)
    rng = np.random.default_rng(56)
    srv = knn.Server(g, k, 1024, grow_headroom_bytes=8 << 30)
    n, used, nreq = n0, 0, 0
    inflight = []
    mark, t_mark, q_lat = n0, time.perf_counter(), []
    t_start = t_mark
    while n < n_end and time.perf_counter() - t_start < 1800.0:   # at most half an hour
        while len(inflight) < 8:
            if nreq % 20 == 19:
                q = mix.sample(1, 1_000_000 + nreq)
                inflight.append((srv.submit(knn.KNN_REQ_QUERY, q), 1, knn.KNN_REQ_QUERY))
            else:
                if used + req > pool.shape[0]:
                    used = 0
                inflight.append((srv.submit(knn.KNN_REQ_INSERT, pool[used:used + req]), req,
                                 knn.KNN_REQ_INSERT))
                used += req
            nreq += 1
        rid, m, kind = inflight.pop(0)
        _, _, info = srv.wait(rid, m, kind)
        if kind == knn.KNN_REQ_INSERT:
            n += m
        else:
            q_lat.append(info["latency_ms"])
        if n - mark >= 200_000 or n >= n_end:
            now = time.perf_counter()
            st = srv.stats()
            q_lat.sort()
            _exp_line(experiment="growth", n=n, capacity=st["capacity"], grows=st["grows"],
                      inserts_per_s=(n - mark) / (now - t_mark),
                      query_latency_ms_p50=q_lat[len(q_lat) // 2] if q_lat else None,
                      query_latency_ms_max=q_lat[-1] if q_lat else None,
                      seconds=now - t_start)
            mark, t_mark, q_lat = n, now, []
    for rid, m, kind in inflight:
        srv.wait(rid, m, kind)
    srv.close()
    st = g.stats()
    _exp_line(experiment="growth_end", n=st["n"], capacity=st["capacity"], device_bytes=st["device_bytes"],
              seconds=time.perf_counter() - t_start)
    g.close()


def run_batching_experiment(knn, torch, np):
    """The batching pattern: 64 independent graphs of uneven sizes (n
    log-uniform in 1,000 .. 200,000, d = 64 FP32, k = 10, each its own
    10-component mixture with means in [-10, 10]^64, sigma 1) in one arena,
    receiving steps of 16..4,096 items (insert : query = 1 : 1, graphs
    uniform).  The search launch width and step size cap are autotuned on
    query-only steps; then the same 60 steps run with the step's launch
    sequence replayed from a CUDA graph and run directly."""
    from paper_1602_06819_gb300 import inputs
    rng = np.random.default_rng(61)
    G, k, n_steps = 64, 10, 60
    sizes = np.floor(10 ** rng.uniform(3, np.log10(2e5), G)).astype(np.int64)
    mixes = [inputs.Mixture(d=64, components=10, half_width=10.0, sigma=1.0, seed=100 + i) for i in range(G)]
    inits = np.concatenate([mixes[i].sample(int(sizes[i]), 1) for i in range(G)])
    caps = sizes + 4096
    steps, qid = [], 0
    for t in range(n_steps):
        m = int(rng.integers(16, 4097))
        graph = rng.integers(0, G, m).astype(np.int32)
        kind = (rng.random(m) < 0.5).astype(np.int32)
        vecs = np.empty((m, 64), np.float32)
        for gi in np.unique(graph):
            idx = np.flatnonzero(graph == gi)
            vecs[idx] = mixes[gi].sample(idx.size, 1000 + 97 * t + int(gi))
        steps.append((vecs, graph, kind, np.arange(qid, qid + m, dtype=np.uint64)))
        qid += m
    sample_g = rng.integers(0, G, 4096).astype(np.int32)
    sample_v = np.stack([mixes[gi].sample(1, 5_000_000 + i)[0] for i, gi in enumerate(sample_g)])
    sample = (sample_v, sample_g, np.arange(4096, dtype=np.uint64))
    X0 = torch.from_numpy(inits).cuda()
    tuned = None
    for use_graph in (True, False):
        cfg = knn.GraphConfig(dim=64, k=k, depth=2, speedup=4.0, expansion=5.0, max_batch=4096, seed=3)
        t0 = time.perf_counter()
        mg = knn.MultiGraph(cfg, sizes, caps, X0, use_graph=use_graph)
        build_s = time.perf_counter() - t0
        if tuned is None:
            tuned = mg.autotune(sample)
            _exp_line(experiment="batching_autotune", **tuned["best"],
                      tried=[{kk: (round(v) if kk == "items_per_s" else v) for kk, v in r.items()}
                             for r in tuned["tried"]])
        else:
            mg.set_launch(tuned["best"]["search_warps"])
            mg.set_order(tuned["best"]["largest_first"])
        cap = tuned["best"]["step_cap"]
        for vecs, graph, kind, qids in steps[:3]:   # warm-up (and capture)
            mg.step_many(vecs, graph, kind, qids, cap)
        lat, items = [], 0
        t0 = time.perf_counter()
        for vecs, graph, kind, qids in steps[3:]:
            a = time.perf_counter()
            mg.step_many(vecs, graph, kind, qids, cap)
            lat.append((time.perf_counter() - a) * 1e3)
            items += len(graph)
        wall = time.perf_counter() - t0
        total_n = sum(mg.size(i)[0] for i in range(G))
        mg.close()
        lat.sort()
        _exp_line(experiment="batching", graphs=G, d=64, k=k, sizes_min=int(sizes.min()), sizes_max=int(sizes.max()),
                  nodes_total=int(total_n), use_cuda_graph=use_graph, search_warps=tuned["best"]["search_warps"],
                  step_cap=cap, steps=len(lat), items_per_s=items / wall, step_ms_p50=lat[len(lat) // 2],
                  step_ms_p99=lat[-1], mean_items_per_step=items / len(lat), build_s=build_s)


def run_tail_experiment(knn, torch, np):
    """What bounds a search launch: per-insert counters of one 1,024-point
    insert batch (every insert spends the same budget, but the dependent
    climb steps and kept restarts vary widely), and the time of query
    launches of 64, 256 and 1,024 queries -- a launch lasts as long as its
    slowest search.  On the d = 128 workload (100,000 points, FP32) and the
    precision workload (1,000,000 points, d = 96, k = 20, BF16 screening)."""
    from paper_1602_06819_gb300 import inputs
    names = ("search_evals", "update_evals", "restarts", "discarded", "moves", "adjacency_reads",
             "draws")
    B = 1024  # insert batches of 1,024 on both workloads
    for W, storage in ((inputs.PLAIN_D128, knn.KNN_STORAGE_FP32),
                       (inputs.PRECISION_D96, knn.KNN_STORAGE_BF16)):
        X0 = torch.from_numpy(W.initial()).cuda()
        Xs = torch.from_numpy(W.mixture.sample(3 * B, W.seed_stream)).cuda()
        Q = torch.from_numpy(W.queries(1024)).cuda()
        cfg = knn.GraphConfig(dim=W.mixture.d, k=W.k, depth=2, storage=storage, speedup=4.0,
                              expansion=W.expansion, rescore_mult=4, max_batch=B,
                              seed=W.seed_search, capacity=W.n_init + 3 * B)
        g = knn.Graph(cfg, X0)
        g.set_timing(True)
        for i in range(3):
            g.insert(Xs[i * B:(i + 1) * B])
        search_ms = g.last_timing()["search"]
        ctr = np.empty((B, 8), np.int64)
        g.counters(ctr)
        pct = {nm: [int(np.percentile(ctr[:, c], p)) for p in (0, 50, 90, 99, 100)]
               for c, nm in enumerate(names)}
        pct["kept_restarts"] = [int(np.percentile(ctr[:, 2] - ctr[:, 3], p)) for p in (0, 50, 90, 99, 100)]
        ids = torch.empty((1024, W.k), dtype=torch.int64, device="cuda")
        launch_ms = {}
        for m in (64, 256, 1024):
            g.query(Q[:m], W.k, 0, ids[:m])
            launch_ms[m] = g.last_timing()["search"]
        g.close()
        _exp_line(experiment="tail", workload=W.name, storage={0: "fp32", 1: "bf16"}[storage], batch=B,
                  n=W.n_init + 2 * B,
                  insert_batch_search_ms=search_ms, per_insert_percentiles_0_50_90_99_100=pct,
                  query_launch_ms=launch_ms)
        del X0, Xs, Q
        torch.cuda.empty_cache()


def main():
    args = parse_args()
    W = pick_workload(args)
    if args.impl == "reference":
        run_reference(args, W)
        return
    if args.experiment:
        import numpy as np
        import torch
        from paper_1602_06819_gb300 import build as kbuild
        kbuild.build()
        from paper_1602_06819_gb300 import knn
        torch.cuda.set_device(0)
        {"search": run_search_experiment, "depth": run_depth_experiment,
         "partitions": run_partition_experiment, "serving": run_serving_experiment,
         "batching": run_batching_experiment, "tail": run_tail_experiment,
         "growth": run_growth_experiment, "distributed": run_distributed_experiment}[args.experiment](
            knn, torch, np)
        return

    import numpy as np
    import torch
    from paper_1602_06819_gb300 import build as kbuild
    kbuild.build()
    from paper_1602_06819_gb300 import knn

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    K, Wm, B = args.steps, args.warmup, W.batch
    n_stream = (K + Wm) * B
    X0 = torch.from_numpy(W.initial()).cuda()
    order_ms = None
    if args.order == "kmedoids":
        # Algorithm 4 as a node ordering: the clusters become contiguous id ranges
        perm = torch.empty(W.n_init, dtype=torch.int64, device="cuda")
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        o0.record()
        knn.knn_balanced_kmedoids(X0, kmedoids_clusters(W.n_init), 1.1, 8, 1, W.seed_search, order=perm)
        o1.record()
        torch.cuda.synchronize()
        order_ms = o0.elapsed_time(o1)
        X0 = X0[perm].contiguous()
    # one fixed stream per rank; a run inserts its prefix
    Xs_host = W.mixture.sample(max(n_stream, W.n_insert), W.seed_stream + 1000 * rank)[:n_stream]
    Xs = torch.from_numpy(Xs_host).cuda()
    capacity = W.n_init + n_stream
    storage = {"fp32": knn.KNN_STORAGE_FP32, "bf16": knn.KNN_STORAGE_BF16,
               "fp8": knn.KNN_STORAGE_FP8_E4M3}[args.storage]
    cfg = knn.GraphConfig(dim=W.mixture.d, k=W.k, depth=args.depth, storage=storage,
                          speedup=args.speedup, expansion=args.expansion,
                          rescore_mult=args.rescore_mult, max_batch=B,
                          seed=W.seed_search + rank, capacity=capacity)

    # exact initial graph (timed on its own, not part of a step)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    g = knn.Graph(cfg, X0)
    e1.record()
    torch.cuda.synchronize()
    exact_ms = e0.elapsed_time(e1)
    g.set_timing(True)

    for i in range(Wm):
        g.insert(Xs[i * B:(i + 1) * B])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    phases = {p: 0.0 for p in knn.PHASES}
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    st0 = g.stats()
    n_before = st0["n"]
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(K):
        flush.fill_(float(i))
        a, b = ev[i]
        a.record()
        g.insert(Xs[(Wm + i) * B:(Wm + i + 1) * B])
        b.record()
        for p, v in g.last_timing().items():
            phases[p] += v
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    st1 = g.stats()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, inserts = aggregate_replicas(dist, sum(step_ms), K * B, device="cuda")
    value = inserts / (total_ms / 1e3)

    # edge recall and Q of the final graph against its exact graph (Sec. 8.5)
    n_final = st1["n"]
    Xall = torch.cat([X0, Xs[:n_final - W.n_init]])
    exact = torch.empty((n_final, W.k), dtype=torch.int64, device="cuda")
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    x0.record()
    knn.knn_exact_graph(Xall, W.k, exact)
    x1.record()
    torch.cuda.synchronize()
    exact_gt = exact_build_report(W, n_final, x0.elapsed_time(x1), knn.knn_exact_last_info())
    online = torch.empty((n_final, W.k), dtype=torch.int64, device="cuda")
    g.edges(online)
    e_c = edge_recall(torch, online, exact)
    e_c_new = edge_recall(torch, online[W.n_init:], exact[W.n_init:])
    recall = e_c / exact.numel()
    recall_new = e_c_new / ((n_final - W.n_init) * W.k)
    q = quality_q(e_c, W.n_init, n_final - W.n_init, W.k)
    extras = rank == 0 and world == 1 and args.workload == "plain" and not args.no_precision
    queries = guarded("queries", run_query_record, knn, torch, g, W, Xall) if extras else None
    del online, Xall
    seq = sequential_oracle_recall(args, W, n_final - W.n_init) if rank == 0 else None

    # roofline of the dominant kernel (the iGNNS search)
    dp = next(v for v in (16, 32, 64, 96, 128, 256) if W.mixture.d <= v)
    row_bytes = {"fp32": 4 * dp, "bf16": 2 * dp, "fp8": dp + 4}[args.storage]
    d_evals = st1["search_evals"] - st0["search_evals"]
    d_adj = st1["adjacency_reads"] - st0["adjacency_reads"]
    alg_bytes_launch = (d_evals * row_bytes + d_adj * W.k * 4 + K * B * 4 * dp) / K
    search_ms = phases["search"] / K
    achieved = alg_bytes_launch / (search_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    traffic, traffic_src = (profiled_traffic() if (args.workload, args.storage) == ("plain", "fp32")
                            else (None, None))
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    g.close()
    del g

    # end to end through the C ABI with host buffers (fresh graph, same batches)
    e2e = None
    if not args.no_e2e:
        g2 = knn.Graph(cfg, X0)
        Xp = torch.from_numpy(Xs_host).pin_memory()
        ids_h = torch.empty(B, dtype=torch.int64).pin_memory()
        nbrs_h = torch.empty((B, W.k), dtype=torch.int64).pin_memory()
        for i in range(Wm):
            g2.insert(Xp[i * B:(i + 1) * B], ids_h, nbrs_h)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e2e_s = 0.0
        for i in range(K):
            # the same L2 flush as the device-timed steps, outside the clock
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2.insert(Xp[(Wm + i) * B:(Wm + i + 1) * B], ids_h, nbrs_h)
            torch.cuda.synchronize()
            e2e_s += time.perf_counter() - t0
        wall_ms, _ = aggregate_replicas(dist, 1e3 * e2e_s, K * B, device="cuda")
        wall = wall_ms / 1e3
        g2.close()
        e2e = {"value": inserts / wall, "unit": UNIT,
               "h2d_bytes_per_step": B * W.mixture.d * 4,
               "d2h_bytes_per_step": B * W.k * 8}

    sweep = (guarded("speedup_sweep", run_speedup_sweep, knn, torch, cfg, X0, Xs, Wm, K, B, exact, flush)
             if extras else None)
    del exact
    precision = None
    if extras:
        del flush
        torch.cuda.empty_cache()
        precision = guarded("precision", run_precision_record, knn, torch, np, peak, peak_src)

    cpu = None
    n_full_avg = n_before + K * B / 2
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = guarded("cpu_baseline", run_cpu_baseline, args, W, n_full_avg)

    if rank == 0:
        srt = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16+f32", "fp8": "e4m3+f32"}[args.storage],
            "data": "synthetic", "config": workload_config(args, W),
            "recall": recall_record(recall, recall_new, q, n_final, seq),
            "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                           "unit": f"one {B:,}-point insert batch"},
            "evals_per_insert": {"search": d_evals / (K * B),
                                 "update": (st1["update_evals"] - st0["update_evals"]) / (K * B),
                                 "cross": (st1["cross_evals"] - st0["cross_evals"]) / (K * B)},
            "phases_ms_per_step": {p: v / K for p, v in phases.items()},
            "exact_build_ms": exact_ms,
            "order_ms": order_ms,
            "exact_ground_truth": exact_gt,
            "roofline": {"kernel": f"ignns_search_kernel<{args.storage},{dp}>", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs",
                         "traffic": traffic, "traffic_source": traffic_src,
                         "algorithmic_bytes_per_launch": alg_bytes_launch,
                         "launch_ms": search_ms},
            "e2e": e2e,
            "speedup_sweep": sweep,
            "queries": queries,
            "precision": precision,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
