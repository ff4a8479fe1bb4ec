"""Online inserts (Algorithm 1 = iGNNS + Update) on the GPU against the oracle.

* One point per call: the GPU path must reproduce the sequential oracle
  exactly -- same search counters, same Update counters, same neighbour list
  for the new point, and the same whole graph -- up to the first insert whose
  decisions include a near tie within FP32 rounding.
* Batches: the edge recall of the GPU graph against the exact graph must be
  within 0.01 of the sequential oracle's recall on the same stream.
* The full-size launch shapes are in test_gpu_full_size.py.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import cuda_tensor, gather_tol, rel_err
from paper_1602_06819_gb300.inputs import PLAIN_D128, SMALL_D16, Mixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


def make_graph(knn, X0, k, speedup, expansion, seed, capacity, max_batch, depth=2, storage=0,
               nbr_ids=None):
    cfg = knn.GraphConfig(dim=X0.shape[1], k=k, depth=depth, storage=storage, speedup=speedup,
                          expansion=expansion, rescore_mult=4, max_batch=max_batch, seed=seed,
                          capacity=capacity)
    return knn.Graph(cfg, cuda_tensor(X0),
                     nbr_ids=None if nbr_ids is None else cuda_tensor(nbr_ids))


def edges(g, n, k):
    import torch
    ids = torch.empty((n, k), dtype=torch.int64, device="cuda")
    sims = torch.empty((n, k), dtype=torch.float32, device="cuda")
    assert g.edges(ids, sims) == n
    return ids.cpu().numpy(), sims.cpu().numpy()


def oracle_graph(X0, ids, sims, capacity):
    """An oracle graph (Algorithm 1's state) over X0 with the given lists."""
    n, d = X0.shape
    og = oracle.Graph(d, ids.shape[1], capacity)
    og.X[:n] = X0
    og.ids[:n] = ids
    og.sims[:n] = sims
    og.n = n
    return og


def single_point_inserts(knn, og, Xs, speedup, e, seed, depth, min_compared, label):
    """Insert Xs one point at a time on both sides, starting from the oracle
    graph og (restored on the GPU).  After every insert the whole GPU graph
    must equal the oracle's, and the insert's counters and new list must
    match; the comparison stops only where the graphs part at an insert whose
    decisions the oracle flags as a near tie.  Returns the inserts compared."""
    import torch
    n0, k, d = og.n, og.k, og.d
    og.X[n0:n0 + len(Xs)] = Xs
    tol = gather_tol(d)
    g = make_graph(knn, og.X[:n0], k, speedup, e, seed, n0 + len(Xs), 1, depth,
                   nbr_ids=og.ids[:n0])
    compared = 0
    try:
        ctr = np.empty((1, 8), np.int64)
        for i in range(len(Xs)):
            new = n0 + i
            L = oracle.search(og.X, og.ids[:new], Xs[i], k, speedup, e, seed, new, n=new)
            og.ids[new], og.sims[new] = L.ids, L.sims
            u = oracle.update(og.X, new + 1, og.ids, og.sims, new, L.ids, L.sims, depth)
            ambiguous = min(L.margin, u.min_margin) < tol
            ids = torch.empty(1, dtype=torch.int64)
            nbrs = torch.empty((1, k), dtype=torch.int64)
            g.insert(cuda_tensor(Xs[i:i + 1]), ids, nbrs)
            g.counters(ctr)
            got_ids, got_sims = edges(g, new + 1, k)
            same = (list(nbrs[0].numpy()) == list(L.ids) and ctr[0, 0] == L.evals and
                    ctr[0, 1] == u.evals and np.array_equal(got_ids, og.ids[:new + 1]))
            if not same:
                assert ambiguous, f"insert {i} differs from the oracle without a near tie"
                break
            assert ids[0].item() == new
            assert rel_err(got_sims, og.sims[:new + 1]).max() <= 1e-5
            compared += 1
    finally:
        g.close()
        og.n = n0 + compared
    print(f"{label}: {compared} of {len(Xs)} single-point inserts equal the oracle, whole graph")
    assert compared >= min_compared, f"only {compared} inserts compared"
    return compared


@pytest.mark.parametrize("speedup,depth", [(4.0, 2), (20.0, 2), (4.0, 1), (4.0, 3), (8.0, 5)])
def test_single_point_inserts_match_sequential_oracle(knn, speedup, depth):
    """Both sides start from the oracle's exact graph (d = 16)."""
    W = SMALL_D16
    X0, Xs = W.initial(), W.stream(250)
    og = oracle.Graph.exact(X0, W.k, capacity=X0.shape[0] + len(Xs))
    single_point_inserts(knn, og, Xs, speedup, W.expansion, W.seed_search, depth, 50,
                         f"d16 speedup {speedup:g} DEPTH {depth}")


def test_single_point_inserts_d128(knn):
    """d = 128 (the benchmark's dimension): 3,000 initial points of the
    benchmark's mixture, 100 points inserted one at a time."""
    W = PLAIN_D128
    X0 = W.mixture.sample(3000, 71)
    Xs = W.mixture.sample(100, 72)
    og = oracle.Graph.exact(X0, W.k, capacity=3100)
    single_point_inserts(knn, og, Xs, 4.0, W.expansion, W.seed_search, 2, 50, "d128")


def _recall(ids, exact):
    return oracle.correct_edges(ids, exact) / exact.size


@pytest.mark.parametrize("batch,depth", [(64, 2), (256, 2), (256, 3), (128, 4)])
def test_batched_inserts_recall_matches_sequential(knn, batch, depth):
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=11)
    n0, na = 4000, 2048
    X0, Xs = mix.sample(n0, 1), mix.sample(na, 2)
    k, speedup, e, seed = 10, 4.0, 5.0, 4
    X = np.vstack([X0, Xs])
    exact, _, _ = oracle.exact_knn(X, k)
    og = oracle.Graph.exact(X0, k, capacity=n0 + na)
    og.insert_stream(Xs, speedup, e, depth, seed)
    r_seq = _recall(og.ids, exact)

    g = make_graph(knn, X0, k, speedup, e, seed, n0 + na, batch, depth)
    try:
        for b0 in range(0, na, batch):
            g.insert(cuda_tensor(Xs[b0:b0 + batch]))
        got, sims = edges(g, n0 + na, k)
        st = g.stats()
    finally:
        g.close()
    r_gpu = _recall(got, exact)
    assert abs(r_gpu - r_seq) <= 0.01, (r_gpu, r_seq)
    # every list: k distinct valid ids, no self, true similarities, sorted
    assert got.min() >= 0 and not np.any(got == np.arange(n0 + na)[:, None])
    srt = np.sort(got, axis=1)
    assert not np.any(srt[:, 1:] == srt[:, :-1])
    assert np.all(np.diff(sims, axis=1) <= 0)
    for u in np.random.default_rng(0).choice(n0 + na, 40, replace=False):
        want = [oracle.similarity(X[u], X[v]) for v in got[u]]
        assert rel_err(sims[u], want).max() <= 1e-5
    assert st["inserts"] == na and st["update_evals"] <= na * sum(k ** t for t in range(2, depth + 1))


def test_batched_inserts_recall_d128(knn):
    """The benchmark's form at a size the oracle finishes in seconds: 20,000
    initial points of the d = 128 mixture, then 8 batches of 1,024.  Batches
    (C14) search the graph as it stood before the batch, so their lists
    differ from the sequential build's; the edge recall against the exact
    graph, over all lists and over the inserted points' lists alone, must be
    within 0.01 of the sequential oracle's (Algorithm 1, one point at a time)
    on the same stream."""
    W = PLAIN_D128
    n0, na, B = 20_000, 8 * 1024, 1024
    X0, Xs = W.mixture.sample(n0, 81), W.mixture.sample(na, 82)
    k, speedup, e, seed = W.k, 4.0, W.expansion, W.seed_search
    X = np.vstack([X0, Xs])
    og = oracle.Graph.exact(X0, k, capacity=n0 + na)
    o_start = og.ids[:n0].copy()
    og.insert_stream(Xs, speedup, e, 2, seed)
    exact, _, _ = oracle.exact_knn(X, k)
    r_seq = _recall(og.ids, exact)
    r_seq_new = _recall(og.ids[n0:], exact[n0:])

    g = make_graph(knn, X0, k, speedup, e, seed, n0 + na, B, 2, nbr_ids=o_start)
    try:
        for b0 in range(0, na, B):
            g.insert(cuda_tensor(Xs[b0:b0 + B]))
        got, _ = edges(g, n0 + na, k)
    finally:
        g.close()
    r_gpu = _recall(got, exact)
    r_gpu_new = _recall(got[n0:], exact[n0:])
    print(f"d128 batches of {B}: edge recall {r_gpu:.4f} (sequential oracle {r_seq:.4f}); "
          f"inserted lists {r_gpu_new:.4f} (oracle {r_seq_new:.4f})")
    assert abs(r_gpu - r_seq) <= 0.01, (r_gpu, r_seq)
    assert abs(r_gpu_new - r_seq_new) <= 0.01, (r_gpu_new, r_seq_new)


def test_insert_edge_cases(knn):
    """The smallest graph (n = k+1), a ragged last batch, and a full graph."""
    import torch
    mix = Mixture(d=5, components=2, half_width=3.0, sigma=1.0, seed=3)
    X0, Xs = mix.sample(11, 1), mix.sample(45, 2)
    g = make_graph(knn, X0, 10, 2.0, 5.0, 1, capacity=56, max_batch=16)
    try:
        for b0 in (0, 16, 32):
            g.insert(cuda_tensor(Xs[b0:b0 + 16]))
        with pytest.raises(knn.KnnError) as exc:
            g.insert(cuda_tensor(Xs[:1]))
        assert exc.value.status == knn.KNN_ERR_CAPACITY
        with pytest.raises(knn.KnnError):
            g.insert(cuda_tensor(np.zeros((17, 5), np.float32)))
        got, _ = edges(g, 56, 10)
    finally:
        g.close()
    X = np.vstack([X0, Xs])
    assert got.min() >= 0 and got.max() < 56
    exact, _, _ = oracle.exact_knn(X, 10)
    assert _recall(got, exact) > 0.8


@pytest.mark.parametrize("m", [64, 1000])
def test_hub_node_under_contention(knn, m):
    """The lock-free Update under contention: m points of one batch placed
    right next to node w (exhaustive search, so w is in every point's level
    1) all offer themselves to w at once through its atomicExch chain; the
    merged list of w must be the best k of its old list and the m points
    (Algorithm 2's offer rule applied in any order)."""
    import torch
    mix = Mixture(d=32, components=5, half_width=10.0, sigma=1.0, seed=19)
    n0, k = 1500, 10
    X0 = mix.sample(n0, 1)
    o_ids, _, _ = oracle.exact_knn(X0, k)
    w = 777
    rng = np.random.default_rng(5)
    pts = (X0[w] + 0.01 * rng.standard_normal((m, 32))).astype(np.float32)
    g = make_graph(knn, X0, k, 1.0, math.inf, 3, n0 + m, max_batch=m, nbr_ids=o_ids)
    try:
        g.insert(cuda_tensor(pts))
        lists, _ = edges(g, n0 + m, k)
    finally:
        g.close()
    allx = np.concatenate([X0, pts]).astype(np.float64)
    cand = np.concatenate([o_ids[w], np.arange(n0, n0 + m)])
    d = np.linalg.norm(allx[cand] - allx[w], axis=1)
    want = cand[np.lexsort((cand, d))][:k]
    assert list(lists[w]) == list(want)
    # and every new point's own list holds w or points of the batch only
    assert np.all((lists[n0:] == w) | (lists[n0:] >= n0))
