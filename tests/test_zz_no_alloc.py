"""knn_search_noalloc -- the query search for callers that cannot allocate
device memory -- against knn_graph_query_batch on the same graph.

Both entry points run the same iGNNS search; the allocation-free one takes
its temporaries from a fixed array inside the library that every call
shares.  Consecutive calls (of different sizes, and a repeat of the first)
must each return what the graph-handle path returns, so nothing left in the
shared array by one call may leak into the next.  This file is collected
last on purpose; it passes on its own and after the other tests.
"""
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


def test_noalloc_search_matches_query_batch(knn):
    import torch
    mix = Mixture(d=128, components=20, half_width=20.0, sigma=1.0, seed=41)
    n, k = 6000, 10
    X0 = mix.sample(n, 1)
    QA, QB = mix.sample(200, 2), mix.sample(333, 3)
    cfg = knn.GraphConfig(dim=128, k=k, speedup=4.0, expansion=5.0, max_batch=512, seed=9,
                          capacity=n)
    Xd = cuda_tensor(X0)
    g = knn.Graph(cfg, Xd)
    try:
        nbr64 = torch.empty((n, k), dtype=torch.int64, device="cuda")
        assert g.edges(nbr64) == n
        nbr32 = nbr64.to(torch.int32).contiguous()
        for Q, qid in ((QA, 5), (QB, 900), (QA, 5)):
            q = cuda_tensor(Q)
            ref_ids = torch.empty((len(Q), k), dtype=torch.int64, device="cuda")
            ref_sims = torch.empty((len(Q), k), dtype=torch.float32, device="cuda")
            g.query(q, k, qid, ref_ids, ref_sims)
            ids = torch.full((len(Q), k), -7, dtype=torch.int64, device="cuda")
            sims = torch.zeros((len(Q), k), dtype=torch.float32, device="cuda")
            knn.knn_search_noalloc(Xd, nbr32, q, k, 4.0, 5.0, 9, qid, ids, sims)
            torch.cuda.synchronize()
            assert torch.equal(ids, ref_ids)
            assert torch.allclose(sims, ref_sims, rtol=1e-5, atol=0.0)
    finally:
        g.close()


def test_noalloc_search_rejects_what_it_cannot_hold(knn):
    import torch
    mix = Mixture(d=16, components=4, half_width=6.0, sigma=1.0, seed=2)
    X = cuda_tensor(mix.sample(240_000, 1))
    nbr = torch.zeros((240_000, 4), dtype=torch.int32, device="cuda")
    Q = cuda_tensor(mix.sample(1024, 2))
    ids = torch.empty((1024, 4), dtype=torch.int64, device="cuda")
    # above 225,280 nodes the visited sets leave shared memory: 1,024 queries
    # x 240,000 nodes need 30 MB of visited bits, beyond the 16 MiB array
    with pytest.raises(knn.KnnError) as exc:
        knn.knn_search_noalloc(X, nbr, Q, 4, 4.0, 5.0, 1, 0, ids)
    assert exc.value.status == knn.KNN_ERR_CAPACITY
    assert "scratch" in str(exc.value)
    # host buffers are refused: nothing is staged
    with pytest.raises(knn.KnnError) as exc:
        knn.knn_search_noalloc(X, nbr, Q.cpu(), 4, 4.0, 5.0, 1, 0, ids)
    assert exc.value.status == knn.KNN_ERR_INVALID_ARG
    # dimensions that would need padding are refused
    with pytest.raises(knn.KnnError) as exc:
        knn.knn_search_noalloc(X[:, :15].contiguous(), nbr, Q[:, :15].contiguous(), 4, 4.0, 5.0,
                               1, 0, ids)
    assert exc.value.status == knn.KNN_ERR_UNSUPPORTED
    # views that start 4 bytes past a 16-byte boundary (rows are read with
    # 16-byte loads) are refused on the host, before any launch
    Xoff = X.view(-1)[1:1 + 1000 * 16].view(1000, 16)
    Qoff = Q.view(-1)[1:1 + 8 * 16].view(8, 16)
    for rows, q in ((Xoff, Q[:8]), (X[:1000], Qoff)):
        with pytest.raises(knn.KnnError) as exc:
            knn.knn_search_noalloc(rows, nbr[:1000], q, 4, 4.0, 5.0, 1, 0, ids[:8])
        assert exc.value.status == knn.KNN_ERR_INVALID_ARG
        assert "16-byte" in str(exc.value)


def test_noalloc_many_queries_with_visited_sets_on_chip(knn):
    """Up to 225,280 nodes the visited sets stay in shared memory and take no
    scratch: 1,024 queries over 200,000 nodes fit the array (the visited bits
    alone would need 25 MB) and match the graph-handle path."""
    import torch
    mix = Mixture(d=16, components=40, half_width=10.0, sigma=1.0, seed=43)
    n, k = 200_000, 8
    Xd = cuda_tensor(mix.sample(n, 1))
    Q = cuda_tensor(mix.sample(1024, 2))
    cfg = knn.GraphConfig(dim=16, k=k, speedup=8.0, expansion=5.0, max_batch=1024, seed=5,
                          capacity=n)
    g = knn.Graph(cfg, Xd)
    try:
        nbr64 = torch.empty((n, k), dtype=torch.int64, device="cuda")
        assert g.edges(nbr64) == n
        nbr32 = nbr64.to(torch.int32).contiguous()
        ref = torch.empty((1024, k), dtype=torch.int64, device="cuda")
        g.query(Q, k, 77, ref)
        for _ in range(2):
            ids = torch.full((1024, k), -7, dtype=torch.int64, device="cuda")
            knn.knn_search_noalloc(Xd, nbr32, Q, k, 8.0, 5.0, 5, 77, ids)
            torch.cuda.synchronize()
            assert torch.equal(ids, ref)
    finally:
        g.close()
