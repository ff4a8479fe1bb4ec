"""The continuous-batching server (knn_server_*): every request completes,
insert ids are dense, and the mix-determinism rule holds -- a query
replayed alone against the graph of its recorded epoch returns exactly what
it returned in the mix, replaying the insert steps rebuilds the same graph,
and inserts served one request per step reach the mixed run's edge recall
within 0.01."""
import threading

import numpy as np
import pytest

from gpu_util import cuda_tensor
from paper_1602_06819_gb300.inputs import Mixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


D, K, N0 = 32, 10, 3000
MIX = Mixture(d=D, components=12, half_width=10.0, sigma=1.0, seed=31)


def make_graph(knn, capacity, max_batch=256, storage=0):
    cfg = knn.GraphConfig(dim=D, k=K, depth=2, storage=storage, speedup=4.0, expansion=5.0,
                          max_batch=max_batch, seed=5, capacity=capacity)
    return knn.Graph(cfg, cuda_tensor(MIX.sample(N0, 1)))


def requests(n_req, seed):
    """(kind, points) of a seeded mix: 1 insert : 4 queries, 1..64 points."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        kind = 0 if rng.random() < 0.2 else 1
        m = int(rng.integers(1, 65))
        out.append((kind, MIX.sample(m, 1000 + 7 * i + seed)))
    return out


def edges(knn, g, n):
    import torch
    e = torch.empty((n, K), dtype=torch.int64, device="cuda")
    assert g.edges(e) == n
    return e.cpu().numpy()


def serve(knn, g, reqs, threads=4, max_step=256, part_offsets=None):
    """Submit from several client threads, each waiting on its own requests."""
    results = {}
    lock = threading.Lock()
    with knn.Server(g, K, max_step, part_offsets=part_offsets) as srv:
        def client(part):
            mine = []
            for idx in part:
                kind, pts = reqs[idx]
                mine.append((idx, srv.submit(kind, pts)))
            for idx, rid in mine:
                kind, pts = reqs[idx]
                ids, sims, info = srv.wait(rid, pts.shape[0], kind)
                with lock:
                    results[idx] = (rid, ids, sims, info)
        parts = [list(range(t, len(reqs), threads)) for t in range(threads)]
        ts = [threading.Thread(target=client, args=(p,)) for p in parts]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        stats = srv.stats()
    return results, stats


def test_mixed_requests_and_replay(knn):
    import torch
    reqs = requests(120, seed=1)
    n_ins = sum(p.shape[0] for k, p in reqs if k == 0)
    g = make_graph(knn, N0 + n_ins)
    try:
        results, stats = serve(knn, g, reqs)
        final = edges(knn, g, N0 + n_ins)
        assert g.stats()["n"] == N0 + n_ins   # the graph is usable again after the server
    finally:
        g.close()
    assert len(results) == len(reqs) and all(r[3]["status"] == 0 for r in results.values())
    assert stats["requests"] == len(reqs) and stats["inserts"] == n_ins and stats["steps"] >= 2
    new_ids = np.concatenate([results[i][1] for i, (k, _) in enumerate(reqs) if k == 0])
    assert sorted(new_ids.tolist()) == list(range(N0, N0 + n_ins))

    # replay: the insert steps in step order (a step packs its inserts in
    # request order), each query alone at its recorded epoch
    steps = {}
    for idx, (kind, pts) in enumerate(reqs):
        rid, ids, sims, info = results[idx]
        steps.setdefault(info["step"], []).append((rid, idx))
    g2 = make_graph(knn, N0 + n_ins)
    try:
        epoch = 0
        for st in sorted(steps):
            members = sorted(steps[st])
            for rid, idx in members:
                kind, pts = reqs[idx]
                if kind != 1:
                    continue
                assert results[idx][3]["epoch"] == epoch
                m = pts.shape[0]
                qids = torch.tensor([(rid << 20) + i for i in range(m)], dtype=torch.int64)
                out = torch.empty((m, K), dtype=torch.int64, device="cuda")
                outs = torch.empty((m, K), dtype=torch.float32, device="cuda")
                g2.query_ids(cuda_tensor(pts), K, qids, out, outs)
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy(), results[idx][1]), f"request {rid}"
                assert np.array_equal(outs.cpu().numpy(), results[idx][2])
            ins = [reqs[idx][1] for rid, idx in members if reqs[idx][0] == 0]
            if ins:
                got = torch.empty(sum(p.shape[0] for p in ins), dtype=torch.int64, device="cuda")
                g2.insert(cuda_tensor(np.concatenate(ins)), got)
                epoch += 1
                want = np.concatenate([results[idx][1] for rid, idx in members if reqs[idx][0] == 0])
                assert np.array_equal(got.cpu().numpy(), want)
        assert np.array_equal(edges(knn, g2, N0 + n_ins), final)
    finally:
        g2.close()


def test_inserts_alone_match_the_mix_in_recall(knn):
    """The same inserts, one request per step (each waited before the next
    is submitted), against the mixed run: the final edge recall against the
    exact graph agrees within 0.01."""
    import torch
    reqs = requests(150, seed=2)
    ins = [(0, p) for k, p in reqs if k == 0]
    n_ins = sum(p.shape[0] for _, p in ins)
    g = make_graph(knn, N0 + n_ins)
    try:
        results, _ = serve(knn, g, reqs)
        mixed = edges(knn, g, N0 + n_ins)
    finally:
        g.close()
    # the requests in the order of the ids the mixed run gave them
    order = np.argsort([results[i][1][0] for i, (k, _) in enumerate(reqs) if k == 0])
    X_all = np.concatenate([MIX.sample(N0, 1)] + [ins[j][1] for j in order])
    exact = torch.empty((N0 + n_ins, K), dtype=torch.int64, device="cuda")
    knn.knn_exact_graph(cuda_tensor(X_all), K, exact)
    exact = exact.cpu().numpy()

    def recall(e):
        return (e[:, :, None] == exact[:, None, :]).any(-1).mean()

    g = make_graph(knn, N0 + n_ins)
    try:
        with knn.Server(g, K, 256) as srv:
            for j in order:
                _, pts = ins[j]
                srv.wait(srv.submit(0, pts), pts.shape[0], 0)
        alone = edges(knn, g, N0 + n_ins)
    finally:
        g.close()
    # the alone run inserted the requests in the mixed run's id order, so both
    # graphs give every point the same id
    assert abs(recall(mixed) - recall(alone)) <= 0.01


def test_capacity_refusal(knn):
    g = make_graph(knn, N0 + 10)
    try:
        with knn.Server(g, K, 64) as srv:
            big = MIX.sample(20, 5)
            rid = srv.submit(0, big)
            with pytest.raises(knn.KnnError):
                srv.wait(rid, 20, 0)
            small = MIX.sample(10, 6)
            ids, _, info = srv.wait(srv.submit(0, small), 10, 0)
            assert info["status"] == 0 and list(ids) == list(range(N0, N0 + 10))
            q = MIX.sample(5, 7)
            ids, sims, info = srv.wait(srv.submit(1, q), 5, 1)
            assert info["status"] == 0 and ids.shape == (5, K) and info["epoch"] == 1
    finally:
        g.close()


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_reserve_keeps_the_graph(knn, storage):
    """Growing a graph mid-stream (knn_graph_reserve) changes nothing the
    method computes, for each searched copy (FP32, BF16, FP8 with its row
    scales): the same inserts give the same lists as a graph created with
    the larger capacity."""
    pts = MIX.sample(300, 41)
    lists = []
    for grow in (False, True):
        g = make_graph(knn, N0 + (100 if grow else 300), storage=storage)
        try:
            g.insert(cuda_tensor(pts[:100]))
            if grow:
                g.reserve(N0 + 300)
                assert g.stats()["capacity"] == N0 + 300
            g.insert(cuda_tensor(pts[100:200]))
            g.insert(cuda_tensor(pts[200:]))
            lists.append(edges(knn, g, N0 + 300))
        finally:
            g.close()
    assert np.array_equal(lists[0], lists[1])


def test_server_grows_the_graph_within_free_memory(knn):
    """Admission by free device memory: with a headroom set, inserts beyond
    the graph's capacity grow it (every request completes, ids stay dense,
    the graph equals a replay of the steps on a graph sized for them from the
    start); with a headroom larger than the device's memory no growth is
    possible and such inserts fail with KNN_ERR_OOM while the rest go on."""
    import torch
    reqs = requests(80, seed=3)
    n_ins = sum(p.shape[0] for k, p in reqs if k == 0)
    g = make_graph(knn, N0 + 20)
    try:
        results = {}
        with knn.Server(g, K, 256, grow_headroom_bytes=256 << 20) as srv:
            rids = [(i, srv.submit(kind, pts)) for i, (kind, pts) in enumerate(reqs)]
            for i, rid in rids:
                kind, pts = reqs[i]
                results[i] = srv.wait(rid, pts.shape[0], kind)
            stats = srv.stats()
        final = edges(knn, g, N0 + n_ins)
    finally:
        g.close()
    assert all(r[2]["status"] == 0 for r in results.values())
    assert stats["grows"] >= 1 and stats["capacity"] >= N0 + n_ins
    new_ids = np.concatenate([results[i][0] for i, (k, _) in enumerate(reqs) if k == 0])
    assert sorted(new_ids.tolist()) == list(range(N0, N0 + n_ins))
    steps = {}
    for i, (kind, _) in enumerate(reqs):
        if kind == 0:
            steps.setdefault(results[i][2]["step"], []).append(i)
    g2 = make_graph(knn, N0 + n_ins)
    try:
        for st in sorted(steps):
            g2.insert(cuda_tensor(np.concatenate([reqs[i][1] for i in sorted(steps[st])])))
        assert np.array_equal(edges(knn, g2, N0 + n_ins), final)
    finally:
        g2.close()

    free, total = torch.cuda.mem_get_info()
    g = make_graph(knn, N0 + 10)
    try:
        with knn.Server(g, K, 64, grow_headroom_bytes=2 * total) as srv:
            rid = srv.submit(0, MIX.sample(20, 5))
            with pytest.raises(knn.KnnError) as exc:
                srv.wait(rid, 20, 0)
            assert exc.value.status == knn.KNN_ERR_OOM
            ids, _, info = srv.wait(srv.submit(0, MIX.sample(10, 6)), 10, 0)
            assert info["status"] == 0 and list(ids) == list(range(N0, N0 + 10))
            assert srv.stats()["grows"] == 0
    finally:
        g.close()


def test_partitioned_queries_alone_match_the_mix(knn):
    """A server whose queries run the partitioned search (Algorithm 3) over
    three node ranges of the initial graph, the last one stretched over the
    nodes inserted since: every query replayed alone
    (knn_graph_query_partitioned_ids) against the graph of its recorded
    epoch, with the parts of that epoch, returns exactly what it returned in
    the mix."""
    import torch
    reqs = requests(100, seed=5)
    n_ins = sum(p.shape[0] for k, p in reqs if k == 0)
    offs = np.array([0, 1000, 2000, N0], np.int64)
    g = make_graph(knn, N0 + n_ins)
    try:
        results, stats = serve(knn, g, reqs, part_offsets=offs)
    finally:
        g.close()
    assert all(r[3]["status"] == 0 for r in results.values())
    steps = {}
    for idx in range(len(reqs)):
        steps.setdefault(results[idx][3]["step"], []).append(idx)
    g2 = make_graph(knn, N0 + n_ins)
    try:
        n = N0
        compared = 0
        for st in sorted(steps):
            members = sorted(steps[st], key=lambda i: results[i][0])
            for idx in members:
                kind, pts = reqs[idx]
                if kind != 1:
                    continue
                rid = results[idx][0]
                m = pts.shape[0]
                qids = torch.tensor([(rid << 20) + i for i in range(m)], dtype=torch.int64)
                out = torch.empty((m, K), dtype=torch.int64, device="cuda")
                outs = torch.empty((m, K), dtype=torch.float32, device="cuda")
                epoch_offs = offs.copy()
                epoch_offs[-1] = n
                g2.query_partitioned_ids(cuda_tensor(pts), K, qids, torch.from_numpy(epoch_offs), out, outs)
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy(), results[idx][1]), f"request {rid}"
                assert np.array_equal(outs.cpu().numpy(), results[idx][2])
                compared += 1
            ins = [reqs[idx][1] for idx in members if reqs[idx][0] == 0]
            if ins:
                g2.insert(cuda_tensor(np.concatenate(ins)))
                n += sum(p.shape[0] for p in ins)
        assert compared == sum(1 for k, _ in reqs if k == 1)
    finally:
        g2.close()
