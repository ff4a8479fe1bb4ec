"""Several graphs in one arena (knn_multi_*): a mixed step of inserts and
queries over graphs of uneven sizes must leave every graph exactly as a
knn_graph given the same items would -- query results (ids and
similarities), new ids and final lists bit-identical -- with the launch
sequence run directly and replayed from a CUDA graph, for FP32 and for BF16
screening, with one warp per item and with a persistent search launch that
takes the items of the largest graphs first."""
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


D, K = 64, 10
SIZES = [300, 1000, 150, 2000, 700]
CAPS = [700, 1600, 400, 2500, 1200]


def mixtures():
    return [Mixture(d=D, components=6, half_width=10.0, sigma=1.0, seed=40 + i) for i in range(len(SIZES))]


def steps(mixes, n_steps, seed):
    """Per step: vecs, graph, kind, query ids of a random mix of items."""
    rng = np.random.default_rng(seed)
    out, qid = [], 0
    for t in range(n_steps):
        m = int(rng.integers(1, 200))
        graph = rng.integers(0, len(mixes), m).astype(np.int32)
        kind = (rng.random(m) < 0.6).astype(np.int32)  # 1 = query
        vecs = np.stack([mixes[gi].sample(1, 10_000 * t + i)[0] for i, gi in enumerate(graph)])
        qids = np.arange(qid, qid + m, dtype=np.uint64)
        qid += m
        out.append((vecs.astype(np.float32), graph, kind, qids))
    return out


@pytest.mark.parametrize("storage,use_graph,largest_first,warps", [
    (0, True, False, 0), (0, False, False, 0), (1, True, False, 0),
    (0, True, True, 64), (1, False, True, 64)])   # persistent searches, largest graphs first
def test_multi_graph_step_equals_single_graphs(knn, storage, use_graph, largest_first, warps):
    import torch
    mixes = mixtures()
    inits = [mixes[i].sample(SIZES[i], 1) for i in range(len(SIZES))]
    cfg = knn.GraphConfig(dim=D, k=K, depth=2, storage=storage, speedup=4.0, expansion=5.0,
                          rescore_mult=4, max_batch=256, seed=7)
    mg = knn.MultiGraph(cfg, SIZES, CAPS, cuda_tensor(np.concatenate(inits)), use_graph=use_graph)
    mg.set_launch(warps)
    mg.set_order(largest_first)
    singles = []
    for i in range(len(SIZES)):
        c = knn.GraphConfig(dim=D, k=K, depth=2, storage=storage, speedup=4.0, expansion=5.0,
                            rescore_mult=4, max_batch=256, seed=7, capacity=CAPS[i])
        singles.append(knn.Graph(c, cuda_tensor(inits[i])))
    try:
        for i, g in enumerate(singles):   # the initial graphs agree
            e = torch.empty((SIZES[i], K), dtype=torch.int64, device="cuda")
            g.edges(e)
            assert np.array_equal(mg.edges(i), e.cpu().numpy())
        for vecs, graph, kind, qids in steps(mixes, 6, seed=3 if storage == 0 else 4):
            out, sims = mg.step(vecs, graph, kind, qids, with_sims=True)
            for i, g in enumerate(singles):
                q = np.flatnonzero((graph == i) & (kind == 1))
                ins = np.flatnonzero((graph == i) & (kind == 0))
                if q.size:   # queries see the graph before the step
                    ids = torch.empty((q.size, K), dtype=torch.int64, device="cuda")
                    sv = torch.empty((q.size, K), dtype=torch.float32, device="cuda")
                    g.query_ids(cuda_tensor(vecs[q]), K, torch.as_tensor(qids[q].astype(np.int64)), ids, sv)
                    torch.cuda.synchronize()
                    assert np.array_equal(out[q], ids.cpu().numpy()), f"graph {i} queries"
                    assert np.array_equal(sims[q], sv.cpu().numpy())
                if ins.size:
                    new = torch.empty(ins.size, dtype=torch.int64, device="cuda")
                    g.insert(cuda_tensor(vecs[ins]), new)
                    torch.cuda.synchronize()
                    assert np.array_equal(out[ins, 0], new.cpu().numpy()), f"graph {i} inserts"
        for i, g in enumerate(singles):
            n, cap = mg.size(i)
            e = torch.empty((n, K), dtype=torch.int64, device="cuda")
            assert g.edges(e) == n and cap == CAPS[i]
            assert np.array_equal(mg.edges(i), e.cpu().numpy()), f"graph {i} lists"
    finally:
        mg.close()
        for g in singles:
            g.close()


def test_multi_graph_capacity(knn):
    mixes = mixtures()
    cfg = knn.GraphConfig(dim=D, k=K, max_batch=64, seed=7)
    sizes, caps = [50, 60], [55, 70]
    inits = np.concatenate([mixes[0].sample(50, 1), mixes[1].sample(60, 1)])
    with knn.MultiGraph(cfg, sizes, caps, inits) as mg:
        vecs = mixes[0].sample(6, 2)
        with pytest.raises(knn.KnnError):
            mg.step(vecs, np.zeros(6, np.int32), np.zeros(6, np.int32))
        out, _ = mg.step(vecs[:5], np.zeros(5, np.int32), np.zeros(5, np.int32))
        assert list(out[:, 0]) == [50, 51, 52, 53, 54] and mg.size(0) == (55, 55)
