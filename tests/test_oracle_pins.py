"""Pins of the FP64 oracle to facts other than itself: published generator
outputs, hand-traced worked examples (tests/golden), closed forms, special
cases that reduce to exhaustive search, an independent library route for the
exact graph, and invariants of Algorithm 2.  No GPU."""
import math

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from conftest import read_golden
from paper_1602_06819_gb300.inputs import Mixture

# --------------------------------------------------------------------------
# generator
# --------------------------------------------------------------------------


def test_splitmix64_published_outputs(orc):
    for ln in read_golden("splitmix64.txt"):
        seed, j, out = (int(t) for t in ln.split())
        assert orc.splitmix64_output(seed, j) == out


def test_search_key_from_published_outputs(orc):
    """The restart key of (seed, stream) is mix(seed XOR mix(stream)), mix(v)
    being output 0 of the generator started at v.  With the published outputs
    mix(0) and mix(1234567), two keys follow without computing SplitMix64:
    key(mix(0) XOR 1234567, 0) = mix(1234567) and key(mix(1234567), 1234567)
    = mix(0)."""
    pub = {(int(a), int(b)): int(c) for a, b, c in (ln.split() for ln in read_golden("splitmix64.txt"))}
    mix0, mix1234567 = pub[(0, 0)], pub[(1234567, 0)]
    assert orc.search_key(mix0 ^ 1234567, 0) == mix1234567
    assert orc.search_key(mix1234567, 1234567) == mix0


def test_draw_closed_forms(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        key = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        j = int(rng.integers(0, 10**6))
        x = orc.splitmix64_output(key, j)
        # n = 2^b: the draw is the top b bits of x
        for b in (1, 7, 20, 31):
            assert orc.draw(key, j, 1 << b) == x >> (64 - b)
        # any n: 0 <= r < n and r = floor(x * n / 2^64) in exact integers
        n = int(rng.integers(1, 5_000_000))
        r = orc.draw(key, j, n)
        assert 0 <= r < n and r == (x * n) >> 64


def test_draws_are_roughly_uniform(orc):
    key = orc.search_key(4, 17)
    n = 10
    counts = np.bincount([orc.draw(key, j, n) for j in range(20000)], minlength=n)
    assert counts.min() > 1800 and counts.max() < 2200


# --------------------------------------------------------------------------
# exact graph (Sec. 2.1)
# --------------------------------------------------------------------------


def test_exact_graph_hand_example(orc):
    X = np.array([[0.0], [1.0], [3.0], [6.0], [10.0]], np.float32)
    ids, sims, margin = orc.exact_knn(X, 2)
    for ln in read_golden("exact_line5.txt"):
        t = [int(v) for v in ln.split()]
        u, nb, dist = t[0], t[1:3], t[3:5]
        assert list(ids[u]) == nb
        np.testing.assert_allclose(sims[u], [1.0 / (1.0 + v) for v in dist], rtol=1e-15)


def _exact_by_library(X, k):
    """Independent route: scipy distance matrix + numpy lexsort."""
    D = cdist(X.astype(np.float64), X.astype(np.float64))
    n = X.shape[0]
    out = np.empty((n, k), np.int64)
    for u in range(n):
        sims = 1.0 / (1.0 + D[u])
        order = np.lexsort((np.arange(n), -sims))
        order = order[order != u]
        out[u] = order[:k]
    return out


@pytest.mark.parametrize("n,d,k,seed", [(60, 3, 5, 1), (200, 16, 10, 2), (150, 7, 1, 3),
                                        (31, 128, 30, 4)])
def test_exact_graph_matches_library_route(orc, n, d, k, seed):
    X = np.random.default_rng(seed).standard_normal((n, d)).astype(np.float32)
    ids, sims, _ = orc.exact_knn(X, k)
    np.testing.assert_array_equal(ids, _exact_by_library(X, k))
    # every list: k distinct non-self ids sorted best first, sims recomputed
    for u in range(n):
        assert len(set(ids[u])) == k and u not in ids[u]
        assert np.all(np.diff(sims[u]) <= 0)
        for v, s in zip(ids[u], sims[u]):
            assert s == pytest.approx(1 / (1 + np.linalg.norm(X[u].astype(np.float64) - X[v])),
                                      rel=1e-12)


def test_exact_graph_duplicates_and_row_subset(orc):
    X = np.random.default_rng(5).standard_normal((40, 4)).astype(np.float32)
    X[7] = X[3]
    X[20] = X[3]
    ids, sims, margin = orc.exact_knn(X, 3)
    assert list(ids[3][:2]) == [7, 20] and sims[3][0] == 1.0
    assert list(ids[7][:2]) == [3, 20]
    assert list(ids[20][:2]) == [3, 7]
    rows = np.array([20, 3, 11])
    ids2, sims2, _ = orc.exact_knn(X, 3, rows=rows)
    np.testing.assert_array_equal(ids2, ids[rows])


def test_exact_graph_skips_removed(orc):
    X = np.random.default_rng(6).standard_normal((50, 5)).astype(np.float32)
    removed = np.zeros(50, np.uint8)
    removed[[4, 9, 33]] = 1
    ids, _, _ = orc.exact_knn(X, 6, removed=removed)
    full = _exact_by_library(np.delete(X, [4, 9, 33], axis=0), 6)
    keep = np.array([i for i in range(50) if not removed[i]])
    for row, u in enumerate(keep):
        assert list(ids[u]) == list(keep[full[row]])


# --------------------------------------------------------------------------
# iGNNS (Sec. 3)
# --------------------------------------------------------------------------


def _line_graph_12():
    X = np.arange(12, dtype=np.float32)[:, None]
    nbr = np.array([[1, 2]] + [[i - 1, i + 1] for i in range(1, 11)] + [[10, 9]], np.int64)
    return X, nbr


def test_ignns_hand_traces(orc):
    X, nbr = _line_graph_12()
    q = np.array([8.2], np.float32)
    for ln in read_golden("ignns_line12.txt"):
        head, draws, result, counts = (p.split() for p in ln.split("|"))
        e, speedup = float(head[1]), float(head[2])
        r = orc.search(X, nbr, q, 3, speedup, e, seed=0, stream=0,
                       draws=[int(v) for v in draws])
        assert list(r.ids) == [int(v) for v in result], head[0]
        ev, rs, dc, mv, du = (int(v) for v in counts)
        assert (r.evals, r.restarts, r.discarded, r.moves, r.draws) == (ev, rs, dc, mv, du), head[0]
        assert r.budget == math.floor(12 / speedup)


def test_ignns_hand_trace_scan_order(orc):
    for ln in read_golden("ignns_gaps10.txt"):
        pts, head, draws, result, counts = (p.split() for p in ln.split("|"))
        X = np.array([[float(v)] for v in pts], np.float32)
        nbr, _, _ = orc.exact_knn(X, 3)
        assert nbr.tolist() == [[1, 2, 3], [2, 0, 3], [3, 1, 4], [4, 2, 5], [5, 3, 6],
                                [6, 4, 7], [7, 5, 8], [8, 6, 9], [9, 7, 6], [8, 7, 6]]
        q, k_out, e, speedup = float(head[0]), int(head[1]), float(head[2]), float(head[3])
        r = orc.search(X, nbr, np.array([q], np.float32), k_out, speedup, e, seed=0,
                       stream=0, draws=[int(v) for v in draws])
        assert list(r.ids) == [int(v) for v in result]
        assert (r.evals, r.restarts, r.discarded, r.moves, r.draws) == tuple(int(v) for v in counts)


def test_gnns_hand_trace(orc):
    """GNNS climb (Sec. 2.2, Sec. 3) and the eager climb side by side on a
    hand-traced six-point line."""
    X = np.array([[10.0], [3.0], [1.0], [8.0], [9.0], [9.5]], np.float32)
    nbr = np.array([[5, 1], [2, 3], [1, 3], [1, 4], [3, 5], [4, 0]], np.int64)
    q = np.array([0.0], np.float32)
    for ln in read_golden("gnns_line6.txt"):
        head, draws, result, counts = (p.split() for p in ln.split("|"))
        climb, speedup = head[1], float(head[2])
        r = orc.search(X, nbr, q, 2, speedup, math.inf, seed=0, stream=0,
                       draws=[int(v) for v in draws], climb=climb)
        assert list(r.ids) == [int(v) for v in result], head[0]
        assert (r.evals, r.restarts, r.discarded, r.moves, r.draws) == \
            tuple(int(v) for v in counts), head[0]


def test_gnns_spends_the_budget_and_moves_uphill(orc):
    """On a mixture graph GNNS spends exactly B = floor(n / speedup)
    evaluations (n_live > B), never discards (no expansion test), and returns
    a sorted list."""
    mix = Mixture(d=8, components=6, half_width=5.0, sigma=1.0, seed=4)
    X = mix.sample(400, 1)
    nbr, _, _ = orc.exact_knn(X, 8)
    for i, q in enumerate(mix.sample(10, 2)):
        for speedup in (4.0, 10.0):
            r = orc.search(X, nbr, q, 5, speedup, math.inf, seed=3, stream=i, climb="best")
            assert r.evals == math.floor(400 / speedup) and r.discarded == 0
            assert np.all(np.diff(r.sims) <= 0)


def test_expansion_test_keeps_equality(orc):
    """Sec. 3's expansion test discards a restart whose similarity is below
    s_max / e; one exactly at the bound is kept.  q = 0, e = 2: the first
    restart (x = 1) sets s_max = 1/2, so the bound is 1/4, which x = 3 meets
    exactly (1 / (1 + 3)); x = 3.5 falls below it and x = 2.5 above.  Every
    list points to its own node, so no restart climbs."""
    q = np.array([0.0], np.float32)
    nbr = np.array([[0], [1]], np.int64)
    for x, discarded in ((3.0, 0), (3.5, 1), (2.5, 0)):
        X = np.array([[1.0], [x]], np.float32)
        r = orc.search(X, nbr, q, 2, 1.0, 2.0, seed=0, stream=0, draws=[0, 1])
        assert (r.evals, r.restarts, r.discarded, r.moves) == (2, 2, discarded, 0), x
        assert r.ids.tolist() == [0, 1]


def test_table1_values_follow_its_formula():
    """Table 1 (Sec. 3) as printed: e_h = k / 2^d, e_l = k - e_h, and e_s and
    the speedup k / e_s from e_s = (k - e_h) / (1 + e_h) to the printed two
    decimals."""
    for ln in read_golden("table1_eager.txt"):
        k, d = (int(v) for v in ln.split()[:2])
        e_h, e_l, e_s, speedup = (float(v) for v in ln.split()[2:])
        assert e_h == k / 2**d and e_l == k - e_h
        f = (k - e_h) / (1 + e_h)
        assert abs(f - e_s) < 0.01 and abs(k / f - speedup) < 0.01


def test_eager_climb_spends_table1_evaluations_per_node(orc):
    """The eager climb moves at the first improving neighbour, so with e_h of
    a node's k neighbours more similar to q, placed uniformly among the list
    positions, it computes on average (k + 1) / (e_h + 1) similarities at that
    node: Table 1's e_s = (k - e_h) / (1 + e_h) before the improving one, plus
    that one; k at a local maximum (e_h = 0).  The GNNS climb computes all k.
    Enumerated exactly over every placement: q = 0 on a line, the start node
    at x = 5 (the only restart), improving neighbours at 1..e_h, the others at
    6, 7, ...; every neighbour's list holds only the start node."""
    from itertools import combinations
    q = np.array([0.0], np.float32)
    for k, e_h in ((4, 1), (10, 1), (10, 2), (10, 3), (10, 0), (6, 6)):
        better = [1.0 + i for i in range(e_h)]
        worse = [6.0 + i for i in range(k - e_h)]
        total_eager, total_best, count = 0, 0, 0
        for pos in combinations(range(k), e_h):
            xs, bi, wi = [], iter(better), iter(worse)
            for i in range(k):
                xs.append(next(bi) if i in pos else next(wi))
            X = np.array([[5.0]] + [[x] for x in xs], np.float32)
            nbr = np.full((k + 1, k), -1, np.int64)
            nbr[0] = np.arange(1, k + 1)
            nbr[1:, 0] = 0
            r = orc.search(X, nbr, q, 1, 1.0, math.inf, seed=0, stream=0, draws=[0])
            total_eager += r.evals - 1
            assert r.moves == (1 if e_h else 0)
            g = orc.search(X, nbr, q, 1, 1.0, math.inf, seed=0, stream=0, draws=[0], climb="best")
            total_best += g.evals - 1
            count += 1
        if e_h:
            assert total_eager * (e_h + 1) == (k + 1) * count          # mean (k+1)/(e_h+1)
            assert math.isclose(total_eager / count - 1, (k - e_h) / (1 + e_h))
        else:
            assert total_eager == k * count
        assert total_best == k * count


def test_ignns_exhaustive_special_case(orc):
    """speedup = 1 and no expansion test: every node is evaluated, so iGNNS is
    linear search (Sec. 2.1) and returns the exact k nearest -- with either
    climb."""
    mix = Mixture(d=8, components=5, half_width=5.0, sigma=1.0, seed=3)
    X = mix.sample(300, 1)
    nbr, _, _ = orc.exact_knn(X, 6)
    Q = mix.sample(20, 2)
    for i, q in enumerate(Q):
        r = orc.search(X, nbr, q, 10, 1.0, math.inf, seed=9, stream=i, climb="eager" if i % 2 else "best")
        sims = 1.0 / (1.0 + np.linalg.norm(X.astype(np.float64) - q.astype(np.float64), axis=1))
        expect = np.lexsort((np.arange(300), -sims))[:10]
        assert list(r.ids) == list(expect)
        assert r.evals == 300 and r.discarded == 0
        np.testing.assert_allclose(r.sims, sims[expect], rtol=1e-13)


@pytest.mark.parametrize("speedup,e", [(2, 5.0), (4, 1.2), (7.5, 2.0), (16, math.inf), (50, 5.0)])
def test_ignns_budget_is_exact(orc, speedup, e):
    """The search computes exactly B = floor(n/speedup) similarities (Sec. 3)
    whenever fewer than all live nodes fit in the budget."""
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=5)
    X = mix.sample(1000, 1)
    nbr, _, _ = orc.exact_knn(X, 10)
    for i, q in enumerate(mix.sample(10, 2)):
        r = orc.search(X, nbr, q, 10, speedup, e, seed=1, stream=i)
        assert r.evals == r.budget == max(1, math.floor(1000 / speedup))
        assert len(set(r.ids)) == 10
        assert np.all(np.diff(r.sims) <= 0)
        assert r.restarts >= 1 and r.discarded <= r.restarts


def test_ignns_budget_floor_is_one(orc):
    """A speedup above n still computes one similarity: B = max(1, floor(n/speedup))."""
    X, nbr = _line_graph_12()
    r = orc.search(X, nbr, np.array([8.2], np.float32), 3, 100.0, 2.0, seed=1, stream=2)
    assert r.budget == 1 and r.evals == 1 and r.restarts == 1
    assert r.ids[0] >= 0 and list(r.ids[1:]) == [-1, -1]


def test_ignns_results_are_true_similarities_and_skip_removed(orc):
    mix = Mixture(d=4, components=3, half_width=4.0, sigma=1.0, seed=8)
    X = mix.sample(200, 1)
    nbr, _, _ = orc.exact_knn(X, 5)
    removed = np.zeros(200, np.uint8)
    removed[::3] = 1
    q = mix.sample(1, 2)[0]
    r = orc.search(X, nbr, q, 8, 1.0, math.inf, seed=2, stream=5, removed=removed)
    live = np.flatnonzero(removed == 0)
    sims = 1.0 / (1.0 + np.linalg.norm(X[live].astype(np.float64) - q, axis=1))
    expect = live[np.lexsort((live, -sims))[:8]]
    assert list(r.ids) == list(expect)
    assert r.evals == live.size


def test_ignns_deterministic_per_stream(orc):
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=5)
    X = mix.sample(500, 1)
    nbr, _, _ = orc.exact_knn(X, 10)
    q = mix.sample(1, 2)[0]
    a = orc.search(X, nbr, q, 10, 4, 5.0, seed=1, stream=3)
    b = orc.search(X, nbr, q, 10, 4, 5.0, seed=1, stream=3)
    c = orc.search(X, nbr, q, 10, 4, 5.0, seed=1, stream=4)
    assert list(a.ids) == list(b.ids) and a.evals == b.evals and a.draws == b.draws
    assert a.draws != c.draws or list(a.ids) != list(c.ids) or a.moves != c.moves


def test_rescore_orders_by_exact_similarity(orc):
    X = np.random.default_rng(1).standard_normal((30, 6)).astype(np.float32)
    q = X[0] + 0.01
    cand = np.array([5, 0, 17, 3, -1, 22], np.int64)
    ids, sims, _ = orc.rescore(X, q, cand, 3)
    s = {int(c): 1 / (1 + np.linalg.norm(X[c].astype(np.float64) - q)) for c in cand if c >= 0}
    expect = sorted(s, key=lambda c: (-s[c], c))[:3]
    assert list(ids) == expect


# --------------------------------------------------------------------------
# Update (Algorithm 2)
# --------------------------------------------------------------------------


def test_update_hand_traces(orc):
    X = np.array([[0], [1], [3], [6], [10], [15], [7]], np.float32)
    for ln in read_golden("update_line6.txt"):
        head, lists, counts = (p.split() for p in ln.split("|"))
        depth = int(head[0])
        ids, sims, _ = orc.exact_knn(X[:6], 2)
        nbr_ids = np.full((7, 2), -1, np.int64)
        nbr_sims = np.full((7, 2), -np.inf)
        nbr_ids[:6], nbr_sims[:6] = ids, sims
        L_ids, L_sims = np.array([3, 4]), np.array([0.5, 0.25])
        nbr_ids[6], nbr_sims[6] = L_ids, L_sims
        st = orc.update(X, 7, nbr_ids, nbr_sims, 6, L_ids, L_sims, depth)
        assert nbr_ids.ravel().tolist() == [int(v) for v in lists], depth
        assert (st.evals, st.literal_evals, st.offers_taken) == tuple(int(v) for v in counts)
        # sims stored with the lists stay the true similarities
        for u in range(7):
            for v, s in zip(nbr_ids[u], nbr_sims[u]):
                assert s == pytest.approx(1 / (1 + abs(float(X[u, 0]) - float(X[v, 0]))), rel=1e-15)


@pytest.mark.parametrize("n,d,k,seed", [(80, 3, 4, 1), (300, 16, 10, 2), (120, 32, 7, 3)])
def test_full_update_gives_exact_graph(orc, n, d, k, seed):
    """Adding one point can only displace entries: an exact graph on n points,
    the exact list of the new point, and an offer to every node give the exact
    graph on n+1 points.  This checks Algorithm 2's offer rule against brute
    force."""
    mix = Mixture(d=d, components=4, half_width=6.0, sigma=1.0, seed=seed)
    X = mix.sample(n + 1, seed + 10)
    ids, sims, _ = orc.exact_knn(X[:n], k)
    nbr_ids = np.vstack([ids, np.full((1, k), -1)]).astype(np.int64)
    nbr_sims = np.vstack([sims, np.full((1, k), -np.inf)])
    L_ids, L_sims, _ = orc.exact_knn(X, k, rows=[n])
    nbr_ids[n], nbr_sims[n] = L_ids[0], L_sims[0]
    orc.update(X, n + 1, nbr_ids, nbr_sims, n, L_ids[0], L_sims[0], 2, full=True)
    exact_ids, exact_sims, _ = orc.exact_knn(X, k)
    np.testing.assert_array_equal(nbr_ids, exact_ids)
    np.testing.assert_allclose(nbr_sims, exact_sims, rtol=1e-15)


def test_update_invariants(orc):
    """Update never lowers a list's k-th similarity, keeps lists sorted with k
    distinct non-self ids, and computes at most k^2 new similarities at DEPTH 2
    (k + k^2 counting the level-1 nodes as Algorithm 2 does)."""
    mix = Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=7)
    X = mix.sample(600, 1)
    k = 10
    g = orc.Graph.exact(X[:500], k, capacity=600)
    g.X[500:] = X[500:]
    for new in range(500, 600):
        before = g.sims[:new, k - 1].copy()
        L = g.search(X[new], k, 4, 5.0, 1, new)
        g.ids[new], g.sims[new] = L.ids, L.sims
        st = orc.update(g.X, new + 1, g.ids, g.sims, new, L.ids, L.sims, 2)
        g.n = new + 1
        assert np.all(g.sims[:new, k - 1] >= before)
        assert st.evals <= k * k and st.literal_evals <= k + k * k
    for u in range(600):
        assert len(set(g.ids[u])) == k and u not in g.ids[u]
        assert np.all(np.diff(g.sims[u]) <= 0)


# --------------------------------------------------------------------------
# sequential online build (Algorithm 1)
# --------------------------------------------------------------------------


def test_insert_stream_matches_explicit_steps(orc):
    """Algorithm 1 is iGNNS then Update for each point in turn."""
    mix = Mixture(d=8, components=4, half_width=6.0, sigma=1.0, seed=2)
    X = mix.sample(260, 1)
    a = orc.Graph.exact(X[:200], 6, capacity=260)
    st = a.insert_stream(X[200:], 3, 5.0, 2, seed=11)
    b = orc.Graph.exact(X[:200], 6, capacity=260)
    b.X[200:] = X[200:]
    for new in range(200, 260):
        L = orc.search(b.X, b.ids[:new], X[new], 6, 3, 5.0, 11, new, n=new)
        b.ids[new], b.sims[new] = L.ids, L.sims
        u = orc.update(b.X, new + 1, b.ids, b.sims, new, L.ids, L.sims, 2)
        assert st["search_evals"][new - 200] == L.evals
        assert st["update_evals"][new - 200] == u.evals
    np.testing.assert_array_equal(a.ids, b.ids)


def test_exhaustive_insert_gives_exact_new_list(orc):
    mix = Mixture(d=8, components=4, half_width=6.0, sigma=1.0, seed=4)
    X = mix.sample(151, 1)
    g = orc.Graph.exact(X[:150], 5, capacity=151)
    g.insert_stream(X[150:], 1.0, math.inf, 2, seed=3)
    exact, _, _ = orc.exact_knn(X, 5, rows=[150])
    assert list(g.ids[150]) == list(exact[0])


def test_depth_sweep_recall_grows_then_flattens(orc):
    """Sec. 8.3: deeper updates give better graphs with diminishing returns."""
    mix = Mixture(d=3, components=10, half_width=10.0, sigma=1.0, seed=9)
    X = mix.sample(800, 1)
    exact, _, _ = orc.exact_knn(X, 10)
    rec = {}
    for depth in (1, 2, 3):
        g = orc.Graph.exact(X[:400], 10, capacity=800)
        g.insert_stream(X[400:], 4, 5.0, depth, seed=5)
        rec[depth] = orc.correct_edges(g.ids, exact) / exact.size
    assert rec[1] < rec[2] <= rec[3] + 0.005
    assert rec[3] - rec[2] < rec[2] - rec[1]


# --------------------------------------------------------------------------
# graph quality (Sec. 8.5)
# --------------------------------------------------------------------------


def test_quality_q_hand_values(orc):
    for ln in read_golden("quality_q.txt"):
        n, n_a, k, e_c, q = ln.split()
        assert orc.quality_q(int(e_c), int(n), int(n_a), int(k)) == pytest.approx(float(q),
                                                                                   rel=1e-9)


def test_correct_edges_counts_directed_overlap(orc):
    a = np.array([[1, 2], [0, 2], [0, 1]])
    b = np.array([[2, 1], [2, 0], [1, 3]])
    assert orc.correct_edges(a, b) == 5
    assert orc.correct_edges(a, a) == 6


# --------------------------------------------------------------------------
# screening storage codes
# --------------------------------------------------------------------------


def test_bf16_codes_match_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 30, rng.standard_normal(1000) * 1e-30,
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 3.4e38]]).astype(np.float32)
    codes, deq = orc.quantize_bf16(x)
    t = torch.from_numpy(x).to(torch.bfloat16)
    np.testing.assert_array_equal(codes, t.view(torch.int16).numpy().view(np.uint16))
    np.testing.assert_array_equal(deq, t.float().numpy())


def test_e4m3_codes_hand_values(orc):
    for v, c in [(0.0, 0x00), (1.0, 0x38), (-1.75, 0xBE), (448.0, 0x7E), (500.0, 0x7E),
                 (-1e9, 0xFE), (2.0**-9, 0x01), (2.0**-6, 0x08), (2.0**-10, 0x00),
                 (3 * 2.0**-11, 0x01), (1.0625, 0x38), (1.1875, 0x3A),
                 (0.0625 * 1.0625, 0x18), (464.0 - 1e-3, 0x7E), (470.0, 0x7E), (-479.0, 0xFE)]:
        assert orc.e4m3_code(v) == c, v
    for c in range(256):
        if c & 0x7F == 0x7F:
            continue                       # the two NaN codes
        assert orc.e4m3_code(orc.e4m3_value(c)) == c


def test_e4m3_codes_match_torch_in_range(orc):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.standard_normal(20000),
                        rng.standard_normal(5000) * 1e-3]).astype(np.float32)
    codes = np.array([orc.e4m3_code(float(v)) for v in x], np.uint8)
    t = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(codes, t)


def test_e4m3_rowwise_scale(orc):
    X = np.random.default_rng(7).standard_normal((50, 96)).astype(np.float32) * 20
    X[3] = 0
    codes, scales, deq = orc.quantize_e4m3(X)
    amax = np.abs(X).max(1)
    np.testing.assert_array_equal(scales[amax > 0], (amax[amax > 0] / np.float32(448)).astype(np.float32))
    assert scales[3] == 1.0 and np.all(deq[3] == 0)
    # the largest element of every row maps to +-448 exactly
    for r in range(50):
        if amax[r] > 0:
            assert np.abs(deq[r]).max() == pytest.approx(amax[r], rel=2e-7)
    # relative error of E4M3 is at most 2^-4 of the value (3 mantissa bits)
    big = np.abs(X) > scales[:, None] * 2.0**-6
    assert np.all(np.abs(deq - X)[big] <= np.abs(X)[big] * 2.0**-4 * 1.0001)


# ---------------------------------------------------------------------------
# balanced k-medoids (Sec. 6, Algorithm 4)
# ---------------------------------------------------------------------------

def test_kmedoids_hand_trace(orc):
    X = np.array([[0.0], [1.0], [2.0], [10.0]], np.float32)
    for ln in read_golden("kmedoids_line4.txt"):
        step, med, imb, want = (p.split() for p in ln.split("|"))
        med = [int(v) for v in med]
        imb = float(imb[0])
        labels, _ = orc.kmedoids_assign(X, med, imb, 1)
        if step[0] == "assign":
            assert labels.tolist() == [int(v) for v in want]
        else:
            new = [orc.kmedoids_medoid(X, np.flatnonzero(labels == m))[0] for m in range(len(med))]
            assert new == [int(v) for v in want]


def test_kmedoids_linear_penalty_hand_trace(orc):
    X = np.array([[0.0], [1.0], [10.0], [3.0]], np.float32)
    for ln in read_golden("kmedoids_penalty4.txt"):
        med, imb, want = (p.split() for p in ln.split("|"))
        labels, _ = orc.kmedoids_assign(X, [int(v) for v in med], float(imb[0]), 1)
        assert labels.tolist() == [int(v) for v in want]


def test_kmedoids_init_draws_distinct_nodes(orc):
    """p = n: the initial medoids are every node once, whatever the seed."""
    for seed in range(6):
        assert sorted(orc.kmedoids_init(5, 5, seed=seed).tolist()) == [0, 1, 2, 3, 4]


def test_kmedoids_one_iteration_is_its_steps(orc):
    """iters = 1 is assign (initial medoids), update, assign: Algorithm 4's
    loop against its steps, each pinned by the hand traces above."""
    mix = Mixture(d=4, components=5, half_width=6.0, sigma=1.0, seed=21)
    X = mix.sample(300, 1)
    p, imb, chunks, seed = 5, 1.2, 2, 7
    med = orc.kmedoids_init(300, p, seed=seed)
    labels, _ = orc.kmedoids_assign(X, med, imb, chunks)
    med1 = np.array([orc.kmedoids_medoid(X, np.flatnonzero(labels == m))[0]
                     if np.any(labels == m) else med[m] for m in range(p)], np.int64)
    labels1, _ = orc.kmedoids_assign(X, med1, imb, chunks)
    got_labels, got_med, _ = orc.kmedoids(X, p, imb, chunks, 1, seed=seed)
    assert got_med.tolist() == med1.tolist() and np.array_equal(got_labels, labels1)
    got_labels0, got_med0, _ = orc.kmedoids(X, p, imb, chunks, 0, seed=seed)
    assert got_med0.tolist() == med.tolist() and np.array_equal(got_labels0, labels)


def test_kmedoids_without_penalty_is_nearest_medoid(orc):
    """imbalance = inf makes w = 1: each point goes to its most similar
    medoid, i.e. the nearest one (checked against a direct argmin)."""
    mix = Mixture(d=6, components=5, half_width=5.0, sigma=1.0, seed=8)
    X = mix.sample(500, 1)
    med = orc.kmedoids_init(500, 12, seed=3)
    labels, margins = orc.kmedoids_assign(X, med, math.inf, 4)
    D = np.linalg.norm(X.astype(np.float64)[:, None, :] - X.astype(np.float64)[med][None], axis=2)
    safe = margins > 1e-12
    assert np.array_equal(labels[safe], np.argmin(D, axis=1)[safe])


def test_kmedoids_balance_and_medoid_definition(orc):
    """With imbalance 1.1 no cluster takes more than ceil(capacity) points of
    a chunk; each medoid the update picks minimises the sum of distances to
    its cluster (checked by brute force); the init draws are distinct."""
    mix = Mixture(d=4, components=3, half_width=5.0, sigma=1.0, seed=9)
    n, p, c = 1200, 8, 3
    X = mix.sample(n, 1)
    med = orc.kmedoids_init(n, p, seed=5)
    assert len(set(med.tolist())) == p and med.min() >= 0 and med.max() < n
    labels, _ = orc.kmedoids_assign(X, med, 1.1, c)
    cap = n * 1.1 / (p * c)
    for j in range(c):
        lo, hi = j * n // c, (j + 1) * n // c
        assert np.bincount(labels[lo:hi], minlength=p).max() <= math.ceil(cap)
    Xd = X.astype(np.float64)
    for m in range(p):
        mem = np.flatnonzero(labels == m)
        got, _ = orc.kmedoids_medoid(X, mem)
        sums = np.linalg.norm(Xd[mem][:, None] - Xd[mem][None], axis=2).sum(1)
        assert got == mem[np.argmin(sums)]


def test_kmedoids_iterations(orc):
    """The whole loop: labels use the returned medoids (re-assigning with
    them reproduces the labels), and every cluster is non-empty."""
    mix = Mixture(d=4, components=6, half_width=8.0, sigma=1.0, seed=2)
    X = mix.sample(900, 1)
    labels, med, _ = orc.kmedoids(X, 6, 1.2, 3, 2, seed=11)
    again, _ = orc.kmedoids_assign(X, med, 1.2, 3)
    assert np.array_equal(labels, again)
    assert np.bincount(labels, minlength=6).min() > 0


# ---------------------------------------------------------------------------
# partitioned search (Sec. 5, Algorithm 3)
# ---------------------------------------------------------------------------

def test_partitioned_search_one_part_is_the_search(orc):
    mix = Mixture(d=8, components=5, half_width=5.0, sigma=1.0, seed=3)
    X = mix.sample(400, 1)
    nbr, _, _ = orc.exact_knn(X, 6)
    for i, q in enumerate(mix.sample(5, 2)):
        ids, sims, tot, _ = orc.partitioned_search(X, nbr, q, 5, [0, 400], 4.0, 5.0, seed=2, stream=i)
        r = orc.search(X, nbr, q, 5, 4.0, 5.0, seed=2, stream=i)
        assert list(ids) == list(r.ids) and tot["evals"] == r.evals and tot["moves"] == r.moves


def test_partitioned_search_exhaustive_and_budget(orc):
    """speedup 1 without the expansion test searches every partition
    exhaustively, so the merged list is the exact k nearest whatever the
    partitions; otherwise the parts spend max(1, floor(size / speedup))
    each."""
    mix = Mixture(d=8, components=5, half_width=5.0, sigma=1.0, seed=4)
    X = mix.sample(500, 1)
    nbr, _, _ = orc.exact_knn(X, 6)
    offs = [0, 90, 260, 261, 500]
    Xd = X.astype(np.float64)
    for i, q in enumerate(mix.sample(6, 2)):
        ids, sims, tot, _ = orc.partitioned_search(X, nbr, q, 8, offs, 1.0, math.inf, seed=1, stream=i)
        s = 1.0 / (1.0 + np.linalg.norm(Xd - q.astype(np.float64), axis=1))
        assert list(ids) == list(np.lexsort((np.arange(500), -s))[:8])
        assert tot["evals"] == 500
        _, _, tot, _ = orc.partitioned_search(X, nbr, q, 8, offs, 7.0, 5.0, seed=1, stream=i)
        assert tot["evals"] == sum(max(1, math.floor((b - a) / 7.0)) for a, b in zip(offs, offs[1:]))


def test_partitioned_search_draw_streams(orc):
    """With a budget of one similarity per part, part j evaluates exactly its
    first restart draw of stream s + j 2^56 among its own nodes."""
    X = Mixture(d=4, components=3, half_width=5.0, sigma=1.0, seed=5).sample(300, 1)
    nbr, _, _ = orc.exact_knn(X, 4)
    offs = [0, 100, 220, 300]
    q = X[7] + 0.1
    s0 = (1 << 63) + 42
    ids, _, tot, _ = orc.partitioned_search(X, nbr, q, 3, offs, 1000.0, 5.0, seed=9, stream=s0)
    want = [a + orc.draw(orc.search_key(9, (s0 + j * (1 << 56)) % (1 << 64)), 0, b - a)
            for j, (a, b) in enumerate(zip(offs, offs[1:]))]
    assert sorted(ids.tolist()) == sorted(want) and tot["evals"] == 3


def test_partitioned_search_does_not_leave_its_part(orc):
    """Lists of part 0 that point only into part 1 give part 0 nothing to
    climb to: its search is restarts only."""
    X = Mixture(d=4, components=2, half_width=5.0, sigma=1.0, seed=6).sample(200, 1)
    nbr = np.empty((200, 4), np.int64)
    nbr[:100] = 100 + (np.arange(100)[:, None] * 7 + np.arange(4)) % 100   # part 0 -> part 1
    nbr[100:] = (np.arange(100)[:, None] * 3 + np.arange(4)) % 100 + 100   # part 1 -> itself
    ids, _, tot, _ = orc.partitioned_search(X, nbr, X[3], 5, [0, 100], 4.0, math.inf, seed=3,
                                            stream=11)
    assert tot["moves"] == 0 and tot["restarts"] == tot["evals"] == 25
    assert np.all(ids < 100)


# ---------------------------------------------------------------------------
# partitions by label (Algorithm 3) and the distributed online build
# (Sec. 7, Algorithm 5)
# ---------------------------------------------------------------------------

def test_partitioned_search_labels_one_part_is_the_search(orc):
    mix = Mixture(d=8, components=5, half_width=5.0, sigma=1.0, seed=13)
    X = mix.sample(400, 1)
    nbr, _, _ = orc.exact_knn(X, 6)
    for i, q in enumerate(mix.sample(5, 2)):
        ids, sims, tot, _ = orc.partitioned_search_labels(X, nbr, q, 5, np.zeros(400, np.int32), 1, 4.0, 5.0,
                                                          seed=2, stream=i)
        r = orc.search(X, nbr, q, 5, 4.0, 5.0, seed=2, stream=i)
        assert list(ids) == list(r.ids) and tot["evals"] == r.evals and tot["moves"] == r.moves


def test_partitioned_search_labels_exhaustive(orc):
    """speedup 1 without the expansion test evaluates every node of every
    partition, so the merged list is the exact k nearest whatever the
    (scattered) labels."""
    mix = Mixture(d=8, components=5, half_width=5.0, sigma=1.0, seed=14)
    X = mix.sample(500, 1)
    nbr, _, _ = orc.exact_knn(X, 6)
    labels = np.random.default_rng(1).integers(0, 4, 500).astype(np.int32)
    Xd = X.astype(np.float64)
    for i, q in enumerate(mix.sample(6, 2)):
        ids, _, tot, _ = orc.partitioned_search_labels(X, nbr, q, 8, labels, 4, 1.0, math.inf, seed=1, stream=i)
        s = 1.0 / (1.0 + np.linalg.norm(Xd - q.astype(np.float64), axis=1))
        assert list(ids) == list(np.lexsort((np.arange(500), -s))[:8])
        assert tot["evals"] == 500


def test_partitioned_search_labels_draw_streams(orc):
    """With a budget of one similarity per partition, partition j evaluates
    its member of position draw(key(seed, s + j 2^56), 0, size_j), its members
    taken in id order."""
    X = Mixture(d=4, components=3, half_width=5.0, sigma=1.0, seed=15).sample(300, 1)
    nbr, _, _ = orc.exact_knn(X, 4)
    labels = (np.arange(300) * 7 % 3).astype(np.int32)
    q = X[7] + 0.1
    s0 = 42
    ids, _, tot, _ = orc.partitioned_search_labels(X, nbr, q, 3, labels, 3, 1000.0, 5.0, seed=9, stream=s0)
    want = []
    for j in range(3):
        members = np.flatnonzero(labels == j)
        want.append(members[orc.draw(orc.search_key(9, s0 + j * (1 << 56)), 0, members.size)])
    assert sorted(ids.tolist()) == sorted(want) and tot["evals"] == 3


def test_partitioned_searches_break_ties_between_parts_to_the_lower_id(orc):
    """Two nodes at the same point in different partitions are equally similar
    to q; the merge of the partitions' results keeps the lower id (the order
    of the exact graph, Sec. 2.1).  1-D points, q = 0, exhaustive searches."""
    X = np.array([[1.0], [5.0], [1.0], [7.0]], np.float32)
    nbr, _, _ = orc.exact_knn(X, 2)
    q = np.array([0.0], np.float32)
    # contiguous parts {0, 1} and {2, 3}: nodes 0 and 2 tie at distance 1
    ids, sims, _, margin = orc.partitioned_search(X, nbr, q, 1, [0, 2, 4], 1.0, math.inf, seed=1, stream=0)
    assert ids.tolist() == [0] and sims[0] == 0.5
    ids, _, _, _ = orc.partitioned_search(X, nbr, q, 3, [0, 2, 4], 1.0, math.inf, seed=1, stream=0)
    assert ids.tolist() == [0, 2, 1]
    # label parts {1, 2} and {0, 3}: the tie is between part 1's node 0 and part 0's node 2
    labels = np.array([1, 0, 0, 1], np.int32)
    ids, sims, _, _ = orc.partitioned_search_labels(X, nbr, q, 1, labels, 2, 1.0, math.inf, seed=1, stream=0)
    assert ids.tolist() == [0] and sims[0] == 0.5
    ids, _, _, _ = orc.partitioned_search_labels(X, nbr, q, 4, labels, 2, 1.0, math.inf, seed=1, stream=0)
    assert ids.tolist() == [0, 2, 1, 3]


def test_partitioned_search_labels_is_the_contiguous_search_renumbered(orc):
    """Renumbering the nodes partition by partition (id order within each)
    turns the label partitions into contiguous ones: the two searches agree."""
    mix = Mixture(d=6, components=6, half_width=6.0, sigma=1.0, seed=16)
    X = mix.sample(600, 1)
    nbr, _, _ = orc.exact_knn(X, 8)
    labels = np.random.default_rng(2).integers(0, 5, 600).astype(np.int32)
    perm = np.lexsort((np.arange(600), labels))            # new position -> node
    pos = np.empty(600, np.int64)
    pos[perm] = np.arange(600)
    Xp = X[perm]
    nbr_p = pos[nbr[perm]]
    offs = np.concatenate([[0], np.cumsum(np.bincount(labels, minlength=5))])
    for i, q in enumerate(mix.sample(8, 3)):
        a = orc.partitioned_search_labels(X, nbr, q, 10, labels, 5, 4.0, 5.0, seed=4, stream=i)
        b = orc.partitioned_search(Xp, nbr_p, q, 10, offs, 4.0, 5.0, seed=4, stream=i)
        assert list(a[0]) == list(perm[b[0]]) and a[2] == b[2]


def test_nearest_medoid_hand_example(orc):
    """1-D points 0, 1, 4, 5, 10 with medoids at nodes 0 (x = 0) and 4
    (x = 10): 4 is nearer 0 than 10; 5 lies halfway, and the tie goes to the
    lower position."""
    X = np.array([[0.0], [1.0], [4.0], [5.0], [10.0]], np.float32)
    labels, margins = orc.nearest_medoid(X, [0, 1, 2, 3, 4], [0, 4])
    assert labels.tolist() == [0, 0, 0, 0, 1]
    assert margins[3] == 0.0 and margins[2] > 0.0
    # the margin is the relative gap of the two best similarities 1 / (1 + L2):
    # x = 4 is at distances 4 and 6, so (1/5 - 1/7) / (1/5) = 2/7; x = 0 at 0
    # and 10, so (1 - 1/11) / 1 = 10/11
    assert margins[2] == pytest.approx(2.0 / 7.0, rel=1e-12)
    assert margins[0] == pytest.approx(10.0 / 11.0, rel=1e-12)
    labels, margins = orc.nearest_medoid(X, [3], [4, 0])       # medoid order decides the tie
    assert labels.tolist() == [0]


def test_medoid_recompute_sizes_paper_example(orc):
    for ln in read_golden("medoid_interval.txt"):
        n_last, interval, n_end, *sizes = ln.split()
        got = orc.medoid_recompute_sizes(int(n_last), int(n_end), float(interval))
        assert got == [int(v) for v in sizes]
    assert orc.medoid_recompute_sizes(4000, 8000, 0.0) == []
    # batches of 1,000: the first batch already passes 10 %
    assert orc.medoid_recompute_sizes(4000, 8000, 0.1, batch=1000) == [5000, 6000, 7000, 8000]


def test_distributed_build_one_partition_is_algorithm_1(orc):
    """One partition and no recompute: Algorithm 5 is Algorithm 1."""
    mix = Mixture(d=8, components=6, half_width=8.0, sigma=1.0, seed=17)
    X0, Xs = mix.sample(500, 1), mix.sample(60, 2)
    a = orc.Graph.exact(X0, 6, capacity=560)
    b = orc.Graph.exact(X0, 6, capacity=560)
    a.insert_stream(Xs, 4.0, 5.0, 2, seed=3)
    labels = np.zeros(560, np.int32)
    st = orc.distributed_insert_stream(b, Xs, labels, np.array([0], np.int64), 4.0, 5.0, 2, 3, 0.0)
    assert np.array_equal(a.ids, b.ids) and np.array_equal(a.sims, b.sims)
    assert st["recomputes"] == 0 and not labels.any()


def test_distributed_build_assigns_and_recomputes(orc):
    """Three partitions, 10 % interval: new nodes go to their nearest medoid;
    the recompute count follows the schedule, and after the last recompute
    every medoid is the member with the smallest sum of distances (scipy)."""
    mix = Mixture(d=4, components=3, half_width=8.0, sigma=1.0, seed=18)
    X0 = mix.sample(300, 1)
    Xs = mix.sample(63, 2)                                      # 300 -> 330 -> 363: two recomputes
    g = orc.Graph.exact(X0, 5, capacity=363)
    labels0, medoids, _ = orc.kmedoids(X0, 3, imbalance=1.1, chunks=1, iters=2, seed=4)
    labels = np.zeros(363, np.int32)
    labels[:300] = labels0
    med_before = medoids.copy()
    st = orc.distributed_insert_stream(g, Xs, labels, medoids, 4.0, 5.0, 2, 5, 0.1)
    assert orc.medoid_recompute_sizes(300, 363, 0.1) == [330, 363]
    assert st["recomputes"] == 2
    # inserts 300..329 were assigned with the initial medoids
    want, _ = orc.nearest_medoid(g.X, np.arange(300, 330), med_before)
    assert np.array_equal(labels[300:330], want)
    D = cdist(g.X[:363].astype(np.float64), g.X[:363].astype(np.float64))
    for j in range(3):
        members = np.flatnonzero(labels == j)
        sums = D[np.ix_(members, members)].sum(1)
        assert medoids[j] == members[np.argmin(sums)]


def test_sequential_recall_fixture_is_consistent(orc):
    """tests/golden/sequential_recall_d128.txt (written by the oracle's
    sequential build, Algorithm 1, on the d = 128 workload) against what its
    own columns fix: recall = e_c / (n k) over all lists and over the
    inserted ones, Q of Sec. 8.5 from e_c, and the mean search cost, which
    the budget fixes exactly (every search of n nodes spends floor(n / 4)
    similarities; n = 100,000 + i for insert i)."""
    rows = [ln.split() for ln in read_golden("sequential_recall_d128.txt")]
    assert [int(r[0]) for r in rows] == [13312, 20480, 25600, 100352]
    n0, k = 100_000, 10
    for r in rows:
        c, n, e_all, e_new = (int(x) for x in r[:4])
        rec, rec_new, q, s_ev, u_ev = (float(x) for x in r[4:])
        assert n == n0 + c
        assert rec == e_all / (n * k) and rec_new == e_new / (c * k)
        assert abs(q - orc.quality_q(e_all, n0, c, k)) <= 1e-12
        budget = sum((n0 + i) // 4 for i in range(c)) / c
        assert s_ev == budget
        assert 0 < u_ev <= k * k
