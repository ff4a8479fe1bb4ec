#!/usr/bin/env python3
"""Write sequential_recall_d128.txt: the graph quality that the sequential
online build (Algorithm 1, one point at a time, FP64 oracle) reaches on the
d = 128 workload, at the insert counts a benchmark or test run stops at.

Workload: the exact graph (Sec. 2.1) of the 100,000 initial points of the
100-component mixture (means U[-20, 20]^128, sigma 1), then the 100,352
stream points inserted in order with iGNNS (Sec. 3) at speedup 4, expansion 5,
and Update (Algorithm 2) to DEPTH 2; restart streams are keyed by the new
point's id with seed 4.  At each checkpoint the oracle's exact graph of all
points so far gives the correct edges e_c (Sec. 8.5) over every list and over
the lists of the inserted points alone.

Calls the oracle only (no GPU, no CUDA library).  Runs for about half an
hour on 8 cores (the exact graphs dominate):

    python tests/golden/make_sequential_recall.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1602_06819_gb300.inputs import PLAIN_D128  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sequential_recall_d128.txt")
SPEEDUP, EXPANSION, DEPTH = 4.0, 5.0, 2
# batches of 1,024 that runs stop at: 8 (the d = 128 recall test at n0 = 20,000
# uses its own stream), 13 (10 + 3), 20, 25 (20 + 5), 98 (95 + 3, the default)
CHECKPOINTS = [13 * 1024, 20 * 1024, 25 * 1024, 98 * 1024]


def main():
    W = PLAIN_D128
    k, n0 = W.k, W.n_init
    X0, Xs = W.initial(), W.stream()
    assert Xs.shape[0] == CHECKPOINTS[-1]
    oracle.build()
    t0 = time.time()
    g = oracle.Graph.exact(X0, k, capacity=n0 + Xs.shape[0])
    print(f"exact graph of {n0}: {time.time() - t0:.0f} s", flush=True)
    rows = []
    done, s_ev, u_ev = 0, 0, 0
    for c in CHECKPOINTS:
        t1 = time.time()
        st = g.insert_stream(Xs[done:c], SPEEDUP, EXPANSION, DEPTH, W.seed_search)
        s_ev += int(st["search_evals"].sum())
        u_ev += int(st["update_evals"].sum())
        done = c
        t2 = time.time()
        n = n0 + c
        exact, _, _ = oracle.exact_knn(g.X[:n], k)
        e_all = oracle.correct_edges(g.ids[:n], exact)
        e_new = oracle.correct_edges(g.ids[n0:n], exact[n0:])
        q = oracle.quality_q(e_all, n0, c, k)
        rows.append((c, n, e_all, e_new, e_all / (n * k), e_new / (c * k), q, s_ev / c, u_ev / c))
        print(f"{c} inserts: recall {e_all / (n * k):.4f}, inserted {e_new / (c * k):.4f}, "
              f"inserts {t2 - t1:.0f} s, exact {time.time() - t2:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("# Sequential online build (Algorithm 1, FP64 oracle) on the d = 128 workload:\n"
                "# exact graph (Sec. 2.1) of the 100,000 initial points of the 100-component\n"
                "# mixture (means U[-20,20]^128, sigma 1, mixture seed 21, initial seed 1), then\n"
                "# the first `inserts` points of the 100,352-point stream (seed 2) one at a time:\n"
                f"# iGNNS (Sec. 3) speedup {SPEEDUP:g}, expansion {EXPANSION:g}, restart seed "
                f"{W.seed_search}, stream = new id;\n"
                f"# Update (Algorithm 2) DEPTH {DEPTH}; k = {k}.  e_c = correct edges (Sec. 8.5) "
                "against the exact graph\n"
                "# of all n points; e_c_inserted counts the lists of the inserted points only.\n"
                "# Written by tests/golden/make_sequential_recall.py (oracle only).\n"
                "# inserts n e_c e_c_inserted edge_recall inserted_recall Q "
                "search_evals_per_insert update_evals_per_insert\n")
        for r in rows:
            f.write(f"{r[0]} {r[1]} {r[2]} {r[3]} {r[4]!r} {r[5]!r} {r[6]!r} {r[7]!r} {r[8]!r}\n")
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
