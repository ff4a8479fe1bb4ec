"""Graphs above 225,280 nodes, where a query's visited set (Sec. 3: no
similarity computed twice) and an Update walk's set of seen nodes
(Algorithm 2) no longer fit in shared memory: the search keeps its bitsets in
global memory (set with L2 atomics, read from L2) and Update its seen sets
likewise.  Both paths are held to the same bar as the on-chip ones: bit-exact
ids and counters against the oracle for every query or insert whose
decisions the oracle does not flag as a near tie, and after each single-point
insert the whole graph equal to the oracle's.

Graph: 240,000 points of d = 16 from a 60-component Gaussian mixture (means
in [-10, 10]^16, sigma 1); its lists are the oracle's exact 10-nn lists
within each component (cheap to build, and a valid k-nn graph for the search
whatever the components' overlap).
"""
import numpy as np
import pytest

import oracle
from paper_1602_06819_gb300.inputs import Mixture
from test_gpu_insert import oracle_graph, single_point_inserts
from test_gpu_search import compare

pytestmark = pytest.mark.gpu

N, K = 240_000, 10


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


@pytest.fixture(scope="module")
def clustered():
    mix = Mixture(d=16, components=60, half_width=10.0, sigma=1.0, seed=61)
    X, labels = mix.sample(N, 1, with_labels=True)
    ids = np.full((N, K), -1, np.int64)
    sims = np.full((N, K), -np.inf)
    for c in range(mix.components):
        idx = np.flatnonzero(labels == c)
        ci, cs, _ = oracle.exact_knn(X[idx], K)
        ids[idx] = idx[ci]
        sims[idx] = cs
    return mix, X, ids, sims


def test_graph_is_above_the_shared_memory_limit():
    """The kernels keep 4 queries' (or Update walks') bitsets per block within
    110 KiB of shared memory; at 240,000 nodes they need more."""
    assert 4 * ((N + 31) // 32) * 4 > 110 * 1024 >= 4 * ((225_280 + 31) // 32) * 4


@pytest.mark.parametrize("storage,m,amb", [(0, 64, 5), (1, 32, 3)])
def test_offchip_queries(knn, clustered, storage, m, amb):
    mix, X, ids, _ = clustered
    Q = mix.sample(m, 3)
    compare(knn, X, Q, K, K, 16.0, 5.0, seed=4, storage=storage, o_ids=ids, max_ambiguous=amb,
            label=f"off-chip visited sets, storage {storage}")


def test_offchip_single_point_inserts(knn, clustered):
    """Each insert's Update walk (DEPTH 2) marks its seen nodes in global
    memory; 16 inserts, the whole 240,000-node graph compared after each (the
    oracle flags none of them as a near tie)."""
    mix, X, ids, sims = clustered
    og = oracle_graph(X, ids, sims, N + 16)
    single_point_inserts(knn, og, mix.sample(16, 5), 16.0, 5.0, 4, 2, 16, "off-chip seen sets")


@pytest.fixture(scope="module")
def clustered_d96():
    """The precision workload's form off chip: d = 96, k = 20, 240,000 points
    of a 120-component mixture, lists exact within each component."""
    mix = Mixture(d=96, components=120, half_width=10.0, sigma=1.0, seed=62)
    X, labels = mix.sample(N, 1, with_labels=True)
    ids = np.full((N, 20), -1, np.int64)
    for c in range(mix.components):
        idx = np.flatnonzero(labels == c)
        ci, _, _ = oracle.exact_knn(X[idx], 20)
        ids[idx] = idx[ci]
    return mix, X, ids


@pytest.mark.parametrize("storage,amb", [(0, 11), (1, 24), (2, 41)])
def test_offchip_queries_d96_k20(knn, clustered_d96, storage, amb):
    """FP32 rows, and BF16 / FP8-E4M3 screening with the FP32 re-score of 4k
    candidates; 48 queries, speedup 16.  The FP8 rows' wider rounding bound
    flags most of these far-reaching searches as near ties."""
    mix, X, ids = clustered_d96
    compare(knn, X, mix.sample(48, 3), 20, 20, 16.0, 5.0, seed=4, storage=storage, o_ids=ids,
            max_ambiguous=amb, label=f"off-chip d96 k20, storage {storage}")


def test_offchip_queries_beyond_resident_warps(knn, clustered):
    """With more searches than warps that fit on the GPU at once (4,096
    queries; three blocks of four warps on each SM), the persistent grid takes
    them from a counter, several a warp: ids, similarities and counters equal
    those of the same queries in launches of 256, where every warp takes one."""
    import torch
    from test_gpu_search import make_graph
    mix, X, ids, _ = clustered
    m = 4096
    Q = torch.from_numpy(mix.sample(m, 7)).cuda()
    g = make_graph(knn, X, K, 64.0, 5.0, 4, nbr_ids=ids, max_batch=m)
    try:
        a_ids = torch.empty((m, K), dtype=torch.int64, device="cuda")
        a_sims = torch.empty((m, K), dtype=torch.float32, device="cuda")
        a_ctr = np.empty((m, 8), np.int64)
        g.query(Q, K, 0, a_ids, a_sims)
        g.counters(a_ctr)
        b_ids, b_sims = torch.empty_like(a_ids), torch.empty_like(a_sims)
        b_ctr = np.empty((m, 8), np.int64)
        for q0 in range(0, m, 256):
            g.query(Q[q0:q0 + 256], K, q0, b_ids[q0:q0 + 256], b_sims[q0:q0 + 256])
            g.counters(b_ctr[q0:q0 + 256])
    finally:
        g.close()
    assert torch.equal(a_ids, b_ids) and torch.equal(a_sims, b_sims)
    assert np.array_equal(a_ctr, b_ctr)
