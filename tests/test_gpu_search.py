"""iGNNS queries (Sec. 3) on the GPU against the oracle's sequential search:
for every query whose decisions all have a margin above the FP32 tolerance,
the ids, the similarity count (the budget), the restarts, discards, moves and
draws must be identical.  The queries the oracle flags as near ties are
counted and printed; each case allows exactly the number the oracle flags for
its seeded inputs (the flags depend on the oracle alone).  Covers the FP32, BF16 and FP8-E4M3 searched copies
(FP32 re-score of the best candidates), removed nodes, the exhaustive
special case and the GNNS climb the paper compares against."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import cuda_tensor, gather_tol, rel_err
from paper_1602_06819_gb300.inputs import Mixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


def make_graph(knn, X0, k, speedup, expansion, seed, storage=0, rescore_mult=4, max_batch=256,
               extra=0, nbr_ids=None):
    """A GPU graph over X0: its exact graph built on the GPU, or, given
    nbr_ids, the oracle's lists restored (so both sides search one graph)."""
    cfg = knn.GraphConfig(dim=X0.shape[1], k=k, depth=2, storage=storage, speedup=speedup,
                          expansion=expansion, rescore_mult=rescore_mult, max_batch=max_batch,
                          seed=seed, capacity=X0.shape[0] + extra)
    return knn.Graph(cfg, cuda_tensor(X0),
                     nbr_ids=None if nbr_ids is None else cuda_tensor(nbr_ids))


def graph_edges(g, n, k):
    import torch
    e = torch.empty((n, k), dtype=torch.int64, device="cuda")
    assert g.edges(e) == n
    return e.cpu().numpy()


def run_queries(g, Q, k_out, qid0):
    import torch
    m = Q.shape[0]
    ids = torch.empty((m, k_out), dtype=torch.int64, device="cuda")
    sims = torch.empty((m, k_out), dtype=torch.float32, device="cuda")
    g.query(cuda_tensor(Q), k_out, qid0, ids, sims)
    ctr = np.empty((m, 8), np.int64)
    g.counters(ctr)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), sims.cpu().numpy(), ctr


def oracle_queries(X0, o_ids, Q, k_out, speedup, e, seed, qid0, storage=0, rescore_mult=4,
                   removed=None, climb="eager"):
    """The oracle's side of compare(): per query the expected ids, similarities
    and counters, and whether a decision of it lies within FP32 reach of a
    tie (ambiguous).  Depends on the oracle only."""
    n, d = X0.shape
    rem = None
    if removed is not None:
        rem = np.zeros(n, np.uint8)
        rem[removed] = 1
    if storage == 1:
        _, Xs = oracle.quantize_bf16(X0)
    elif storage == 2:
        _, _, Xs = oracle.quantize_e4m3(X0)
    else:
        Xs = X0
    tol = gather_tol(d, storage)
    out = []
    for i, q in enumerate(Q):
        kt = k_out if storage == 0 else rescore_mult * k_out
        r = oracle.search(Xs, o_ids, q, kt, speedup, e, seed, (1 << 63) + qid0 + i, removed=rem,
                          climb=climb)
        margin = r.margin
        exp_ids, exp_sims = r.ids, r.sims
        if storage != 0:
            exp_ids, exp_sims, m2 = oracle.rescore(X0, q, r.ids, k_out)
            margin = min(margin, m2)
        out.append(dict(ids=exp_ids, sims=exp_sims, ambiguous=margin < tol,
                        counters=(r.evals, r.restarts, r.discarded, r.moves, r.draws)))
    return out


def check_queries(ids, sims, ctr, expected, max_ambiguous, label=""):
    """Unambiguous queries must match the oracle bit for bit (ids, counters)
    and in similarity (1e-5 relative); the ambiguous ones are counted."""
    ambiguous = 0
    for i, ex in enumerate(expected):
        if ex["ambiguous"]:
            ambiguous += 1
            continue
        assert list(ids[i]) == list(ex["ids"]), f"query {i}"
        valid = ex["ids"] >= 0
        assert rel_err(sims[i][valid], ex["sims"][valid]).max() <= 1e-5
        got = tuple(ctr[i][[0, 2, 3, 4, 6]])
        assert got == ex["counters"], f"query {i}: counters {got} != {ex['counters']}"
        assert ctr[i][1] == 0
    print(f"{label}: {len(expected) - ambiguous} of {len(expected)} queries compared bit-exactly, "
          f"{ambiguous} near ties")
    assert ambiguous <= max_ambiguous, f"{ambiguous} of {len(expected)} ambiguous"
    return ambiguous


def compare(knn, X0, Q, k, k_out, speedup, e, seed, storage=0, rescore_mult=4, removed=None,
            max_ambiguous=0, climb="eager", o_ids=None, label="queries"):
    """max_ambiguous: the number of queries the oracle flags as near ties for
    these seeded inputs (it depends on the oracle alone)."""
    n, d = X0.shape
    if o_ids is None:
        o_ids, _, _ = oracle.exact_knn(X0, k)
    g = make_graph(knn, X0, k, speedup, e, seed, storage, rescore_mult, nbr_ids=o_ids,
                   max_batch=max(256, len(Q)))
    try:
        if climb != "eager":
            g.set_search(speedup, e, climb)
        assert np.array_equal(graph_edges(g, n, k), o_ids), "restored lists differ"
        if removed is not None:
            import torch
            g.remove(torch.as_tensor(removed, dtype=torch.int64))
        qid0 = 1000
        ids, sims, ctr = run_queries(g, Q, k_out, qid0)
    finally:
        g.close()
    expected = oracle_queries(X0, o_ids, Q, k_out, speedup, e, seed, qid0, storage, rescore_mult,
                              removed, climb)
    return check_queries(ids, sims, ctr, expected, max_ambiguous, label)


@pytest.mark.parametrize("speedup,e", [(4.0, 5.0), (20.0, 5.0), (8.0, 1.2), (2.0, math.inf)])
def test_queries_small_d16(knn, speedup, e):
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=11)
    X0, Q = mix.sample(1000, 1), mix.sample(96, 3)
    compare(knn, X0, Q, 10, 10, speedup, e, seed=4)


@pytest.mark.parametrize("d,speedup,e,amb", [(16, 4.0, math.inf, 3), (16, 20.0, math.inf, 0),
                                             (16, 8.0, 5.0, 1), (128, 4.0, math.inf, 14)])
def test_queries_gnns_climb(knn, d, speedup, e, amb):
    """GNNS (Sec. 2.2): every unvisited neighbour evaluated, move to the most
    similar; with and without the expansion test."""
    mix = Mixture(d=d, components=10, half_width=10.0 if d == 16 else 20.0, sigma=1.0, seed=11)
    X0, Q = mix.sample(1000 if d == 16 else 3000, 1), mix.sample(96, 3)
    compare(knn, X0, Q, 10, 10, speedup, e, seed=4, climb="best", max_ambiguous=amb)


def test_queries_gnns_climb_screened_and_removed(knn):
    mix = Mixture(d=32, components=8, half_width=10.0, sigma=1.0, seed=5)
    X0, Q = mix.sample(1500, 1), mix.sample(64, 3)
    removed = np.random.default_rng(3).choice(1500, 60, replace=False)
    compare(knn, X0, Q, 8, 8, 4.0, math.inf, seed=2, storage=1, removed=removed, climb="best",
            max_ambiguous=1)


def test_set_search_changes_parameters(knn):
    """Search parameters changed on a live graph take effect on the next
    call: the budget follows the new speedup."""
    mix = Mixture(d=16, components=4, half_width=10.0, sigma=1.0, seed=6)
    X0, Q = mix.sample(600, 1), mix.sample(8, 2)
    g = make_graph(knn, X0, 8, 4.0, 5.0, seed=1)
    try:
        _, _, c1 = run_queries(g, Q, 5, 0)
        g.set_search(10.0, math.inf, "best")
        _, _, c2 = run_queries(g, Q, 5, 0)
        with pytest.raises(knn.KnnError):
            g.set_search(0.0, 5.0, "eager")
    finally:
        g.close()
    assert np.all(c1[:, 0] == 150) and np.all(c2[:, 0] == 60) and np.all(c2[:, 3] == 0)


def test_queries_d128_many_tiles(knn):
    mix = Mixture(d=128, components=20, half_width=20.0, sigma=1.0, seed=21)
    X0, Q = mix.sample(4000, 1), mix.sample(64, 3)
    compare(knn, X0, Q, 10, 10, 4.0, 5.0, seed=4, max_ambiguous=3)


@pytest.mark.parametrize("d,storage,amb", [(200, 0, 1), (256, 1, 7)])
def test_queries_widest_rows(knn, d, storage, amb):
    """The widest rows (padded to 256): a restart's head is 128 bytes of a
    1,024-byte (FP32) or 512-byte (BF16) row, so fewer restarts are settled
    by their partial sums and more take the full second gather."""
    mix = Mixture(d=d, components=10, half_width=20.0, sigma=1.0, seed=23)
    X0, Q = mix.sample(2500, 1), mix.sample(48, 3)
    compare(knn, X0, Q, 10, 10, 4.0, 5.0, seed=4, storage=storage, max_ambiguous=amb)


def test_queries_ragged_dims_and_k_out(knn):
    mix = Mixture(d=3, components=5, half_width=10.0, sigma=1.0, seed=2)
    X0, Q = mix.sample(700, 1), mix.sample(48, 3)
    compare(knn, X0, Q, 8, 5, 3.0, 2.0, seed=9)
    mix = Mixture(d=100, components=6, half_width=10.0, sigma=1.0, seed=3)
    X0, Q = mix.sample(500, 1), mix.sample(32, 3)
    compare(knn, X0, Q, 10, 10, 2.0, 5.0, seed=9, max_ambiguous=1)


def test_exhaustive_queries_are_linear_search(knn):
    """speedup 1 without the expansion test visits every node: the result is
    the exact k-nn of each query (Sec. 2.1's linear search)."""
    mix = Mixture(d=32, components=4, half_width=8.0, sigma=1.0, seed=5)
    X0, Q = mix.sample(300, 1), mix.sample(40, 3)
    compare(knn, X0, Q, 6, 6, 1.0, math.inf, seed=1)


def test_queries_skip_removed_nodes(knn):
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=11)
    X0, Q = mix.sample(1000, 1), mix.sample(48, 3)
    removed = np.random.default_rng(0).choice(1000, 150, replace=False)
    compare(knn, X0, Q, 10, 10, 3.0, 5.0, seed=4, removed=removed, max_ambiguous=1)
    compare(knn, X0, Q[:16], 10, 10, 1.0, math.inf, seed=4, removed=removed)


@pytest.mark.parametrize("storage,amb96,amb16", [(1, 7, 3), (2, 12, 5)])
def test_screening_queries(knn, storage, amb96, amb16):
    """BF16 / FP8-E4M3 screening with an FP32 re-score of 4k candidates
    against the oracle searching the same stored values."""
    mix = Mixture(d=96, components=10, half_width=20.0, sigma=1.0, seed=31)
    X0, Q = mix.sample(2000, 1), mix.sample(48, 3)
    compare(knn, X0, Q, 10, 10, 4.0, 5.0, seed=4, storage=storage, max_ambiguous=amb96)
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=11)
    X0, Q = mix.sample(1000, 1), mix.sample(48, 3)
    compare(knn, X0, Q, 20, 20, 4.0, 5.0, seed=4, storage=storage, rescore_mult=4,
            max_ambiguous=amb16)


def test_restore_keeps_lists_and_checks_ids(knn):
    import torch
    mix = Mixture(d=16, components=4, half_width=6.0, sigma=1.0, seed=2)
    X0 = mix.sample(300, 1)
    o_ids, o_sims, _ = oracle.exact_knn(X0, 7)
    g = make_graph(knn, X0, 7, 4.0, 5.0, 1, nbr_ids=o_ids)
    try:
        ids = torch.empty((300, 7), dtype=torch.int64, device="cuda")
        sims = torch.empty((300, 7), dtype=torch.float32, device="cuda")
        assert g.edges(ids, sims) == 300
        assert np.array_equal(ids.cpu().numpy(), o_ids)
        assert rel_err(sims.cpu().numpy(), o_sims).max() <= 1e-5
    finally:
        g.close()
    for bad in (300, -2):
        b = o_ids.copy()
        b[5, 3] = bad
        with pytest.raises(knn.KnnError) as exc:
            make_graph(knn, X0, 7, 4.0, 5.0, 1, nbr_ids=b)
        assert exc.value.status == knn.KNN_ERR_INVALID_ARG
    b = o_ids.copy()
    b[9, 0] = 9
    with pytest.raises(knn.KnnError):
        make_graph(knn, X0, 7, 4.0, 5.0, 1, nbr_ids=b)


def test_query_results_do_not_depend_on_the_batch(knn):
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=11)
    X0, Q = mix.sample(1000, 1), mix.sample(64, 3)
    g = make_graph(knn, X0, 10, 4.0, 5.0, 4)
    try:
        all_ids, _, _ = run_queries(g, Q, 10, 500)
        for s in (0, 17, 40):
            part, _, _ = run_queries(g, Q[s:s + 9], 10, 500 + s)
            assert np.array_equal(part, all_ids[s:s + 9])
    finally:
        g.close()


# ---------------------------------------------------------------------------
# partitioned search (Sec. 5, Algorithm 3)
# ---------------------------------------------------------------------------

def oracle_partitioned(X0, o_ids, Q, k_out, offs, speedup, e, seed, qid0, storage=0,
                       removed=None, climb="eager"):
    """The oracle's side of compare_partitioned() (Algorithm 3)."""
    n, d = X0.shape
    rem = None
    if removed is not None:
        rem = np.zeros(n, np.uint8)
        rem[removed] = 1
    Xs = X0
    if storage == 1:
        _, Xs = oracle.quantize_bf16(X0)
    elif storage == 2:
        _, _, Xs = oracle.quantize_e4m3(X0)
    tol = gather_tol(d, storage)
    out = []
    for i, q in enumerate(Q):
        kt = k_out if storage == 0 else 4 * k_out
        e_ids, e_sims, tot, margin = oracle.partitioned_search(Xs, o_ids, q, kt, offs, speedup, e, seed,
                                                               (1 << 63) + qid0 + i, removed=rem,
                                                               climb=climb)
        if storage != 0:
            e_ids, e_sims, m2 = oracle.rescore(X0, q, e_ids, k_out)
            margin = min(margin, m2)
        out.append(dict(ids=e_ids, sims=e_sims, ambiguous=margin < tol,
                        counters=(tot["evals"], tot["restarts"], tot["discarded"], tot["moves"],
                                  tot["draws"])))
    return out


def compare_partitioned(knn, X0, Q, k, k_out, speedup, e, seed, offs, storage=0, removed=None,
                        climb="eager", max_batch=256, max_ambiguous=0, label="partitioned"):
    import torch
    n, d = X0.shape
    o_ids, _, _ = oracle.exact_knn(X0, k)
    g = make_graph(knn, X0, k, speedup, e, seed, storage, 4, max_batch=max_batch, nbr_ids=o_ids)
    m = Q.shape[0]
    try:
        if climb != "eager":
            g.set_search(speedup, e, climb)
        if removed is not None:
            g.remove(torch.as_tensor(removed, dtype=torch.int64))
        qid0 = 500
        ids = torch.empty((m, k_out), dtype=torch.int64, device="cuda")
        sims = torch.empty((m, k_out), dtype=torch.float32, device="cuda")
        g.query_partitioned(cuda_tensor(Q), k_out, qid0, torch.as_tensor(offs, dtype=torch.int64), ids, sims)
        ctr = np.empty((m, 8), np.int64)
        g.counters(ctr)
        torch.cuda.synchronize()
        ids, sims = ids.cpu().numpy(), sims.cpu().numpy()
    finally:
        g.close()
    expected = oracle_partitioned(X0, o_ids, Q, k_out, offs, speedup, e, seed, qid0, storage,
                                  removed, climb)
    return check_queries(ids, sims, ctr, expected, max_ambiguous, label)


@pytest.mark.parametrize("d,n,offs,speedup,e,amb", [
    (16, 1000, [0, 250, 500, 750, 1000], 4.0, 5.0, 0),
    (16, 1000, [0, 37, 400, 401, 1000], 2.0, math.inf, 0),   # uneven parts, one of a single node
    (128, 3000, [0, 300, 700, 1100, 1500, 1800, 2300, 2600, 3000], 8.0, 5.0, 2),
])
def test_partitioned_queries(knn, d, n, offs, speedup, e, amb):
    mix = Mixture(d=d, components=10, half_width=10.0 if d == 16 else 20.0, sigma=1.0, seed=14)
    X0, Q = mix.sample(n, 1), mix.sample(64, 3)
    compare_partitioned(knn, X0, Q, 10, 10, speedup, e, seed=4, offs=offs, max_ambiguous=amb)


def test_partitioned_queries_kmedoids_order_screened_removed_gnns(knn):
    """Partitions from the balanced k-medoids ordering of the points, BF16
    screening with FP32 re-score, removed nodes, the GNNS climb, and more
    queries than one launch holds (max_batch 32 with 8 parts: 4 queries a
    launch)."""
    mix = Mixture(d=32, components=8, half_width=10.0, sigma=1.0, seed=15)
    X = mix.sample(2000, 1)
    labels, _, _ = oracle.kmedoids(X, 8, 1.1, 1, 1, seed=3)
    order = np.lexsort((np.arange(2000), labels))
    X0 = np.ascontiguousarray(X[order])
    offs = np.concatenate([[0], np.cumsum(np.bincount(labels, minlength=8))]).tolist()
    Q = mix.sample(20, 3)
    removed = np.random.default_rng(4).choice(2000, 50, replace=False)
    compare_partitioned(knn, X0, Q, 8, 8, 2.0, math.inf, seed=2, offs=offs, storage=1, removed=removed,
                        climb="best", max_batch=32, max_ambiguous=7)


def test_partitioned_one_part_equals_query_batch(knn):
    import torch
    mix = Mixture(d=16, components=6, half_width=10.0, sigma=1.0, seed=16)
    X0, Q = mix.sample(800, 1), mix.sample(32, 2)
    g = make_graph(knn, X0, 8, 4.0, 5.0, seed=3)
    try:
        a, _, ca = run_queries(g, Q, 8, 77)
        b = torch.empty((32, 8), dtype=torch.int64, device="cuda")
        g.query_partitioned(cuda_tensor(Q), 8, 77, torch.tensor([0, 800], dtype=torch.int64), b)
        cb = np.empty((32, 8), np.int64)
        g.counters(cb)
        torch.cuda.synchronize()
        with pytest.raises(knn.KnnError):
            g.query_partitioned(cuda_tensor(Q), 8, 77, torch.tensor([0, 500], dtype=torch.int64), b)
    finally:
        g.close()
    assert np.array_equal(a, b.cpu().numpy()) and np.array_equal(ca, cb)
