"""Exact k-nn graph (Sec. 2.1) on the GPU against the FP64 oracle: ids
bit-exact except rows with a flagged near tie, similarities within 1e-5
relative, at small sizes spanning several tiles with ragged tails, at the
edge cases (n = k+1, k = 1, k = 32, d = 256, d not a multiple of 16), and at
the full 100,000 x 128 size on sampled rows."""
import numpy as np
import pytest

import oracle
from gpu_util import cuda_tensor, exact_tol, rel_err
from paper_1602_06819_gb300.inputs import PLAIN_D128, Mixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


def gpu_exact(knn, X, k):
    import torch
    n = X.shape[0]
    ids = torch.empty((n, k), dtype=torch.int64, device="cuda")
    sims = torch.empty((n, k), dtype=torch.float32, device="cuda")
    knn.knn_exact_graph(cuda_tensor(X), k, ids, sims)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), sims.cpu().numpy()


def check_rows(ids, sims, o_ids, o_sims, margin, tol):
    safe = margin >= tol
    bad = np.flatnonzero(safe & np.any(ids != o_ids, axis=1))
    assert bad.size == 0, f"rows {bad[:10]} differ from the oracle"
    assert rel_err(sims, o_sims).max() <= 1e-5
    return int((~safe).sum())


@pytest.mark.parametrize("n,d,k,comps,seed", [
    (1000, 16, 10, 10, 1),    # the small workload's initial graph
    (777, 3, 5, 4, 2),        # d padded 3 -> 16, n not a multiple of the 64-row tile
    (600, 128, 10, 6, 3),
    (700, 96, 20, 8, 4),      # k = 20 (32-entry row lists)
    (129, 64, 32, 3, 5),      # k = 32, the largest
    (33, 256, 32, 2, 6),      # n = k + 1, the smallest graph; d = 256, the largest
    (65, 100, 1, 2, 7),       # k = 1; d = 100 padded to 128
])
def test_exact_graph_matches_oracle(knn, n, d, k, comps, seed):
    X = Mixture(d=d, components=comps, half_width=10.0, sigma=1.0, seed=seed).sample(n, seed + 100)
    ids, sims = gpu_exact(knn, X, k)
    o_ids, o_sims, margin = oracle.exact_knn(X, k)
    flagged = check_rows(ids, sims, o_ids, o_sims, margin, exact_tol(d))
    assert flagged <= n // 2   # k boundaries per row can each be a near tie


def test_exact_graph_duplicates_tie_to_lower_id(knn):
    X = Mixture(d=16, components=3, half_width=5.0, sigma=1.0, seed=9).sample(200, 1)
    X[50] = X[10]
    X[120] = X[10]
    ids, sims = gpu_exact(knn, X, 4)
    assert list(ids[10][:2]) == [50, 120] and sims[10][0] == 1.0
    assert list(ids[120][:2]) == [10, 50]


def test_exact_graph_full_size_sampled_rows(knn):
    """The 100,000-point, d = 128 initial graph: 48 sampled rows against the
    oracle, and the list invariants on every row."""
    X = PLAIN_D128.initial()
    k = PLAIN_D128.k
    ids, sims = gpu_exact(knn, X, k)
    rows = np.random.default_rng(5).choice(X.shape[0], 48, replace=False)
    o_ids, o_sims, margin = oracle.exact_knn(X, k, rows=rows)
    check_rows(ids[rows], sims[rows], o_ids, o_sims, margin, exact_tol(128))
    n = X.shape[0]
    assert ids.min() >= 0 and ids.max() < n
    assert not np.any(ids == np.arange(n)[:, None])
    srt = np.sort(ids, axis=1)
    assert not np.any(srt[:, 1:] == srt[:, :-1])
    assert np.all(np.diff(sims, axis=1) <= 0)
