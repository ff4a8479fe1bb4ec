"""Exact k-nn graph (Sec. 2.1) on the GPU against the FP64 oracle: ids
bit-exact except rows with a flagged near tie, similarities within 1e-5
relative, at small sizes spanning several tiles with ragged tails, at the
edge cases (n = k+1, k = 1, k = 32, d = 256, d not a multiple of 16), and at
the full 100,000 x 128 size on sampled rows -- on both paths, the CUDA-core
kernel and the tensor-core screening with FP32 settling."""
import numpy as np
import pytest

import oracle
from gpu_util import cuda_tensor, exact_tol, padded, rel_err
from paper_1602_06819_gb300.inputs import PLAIN_D128, Mixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


def gpu_exact(knn, X, k, path="auto"):
    import torch
    n = X.shape[0]
    ids = torch.empty((n, k), dtype=torch.int64, device="cuda")
    sims = torch.empty((n, k), dtype=torch.float32, device="cuda")
    knn.knn_exact_set_path(path)
    try:
        knn.knn_exact_graph(cuda_tensor(X), k, ids, sims)
    finally:
        knn.knn_exact_set_path("auto")
    torch.cuda.synchronize()
    info = knn.knn_exact_last_info()
    if path != "auto":
        assert info["path"] == path
    assert info["n"] == n and info["wait_errors"] == 0
    return ids.cpu().numpy(), sims.cpu().numpy()


def tc_capable(n, d):
    return padded(d) <= 128 and n >= 128


def check_rows(ids, sims, o_ids, o_sims, margin, tol):
    safe = margin >= tol
    bad = np.flatnonzero(safe & np.any(ids != o_ids, axis=1))
    assert bad.size == 0, f"rows {bad[:10]} differ from the oracle"
    assert rel_err(sims, o_sims).max() <= 1e-5
    return int((~safe).sum())


EXACT_CASES = [
    (1000, 16, 10, 10, 1),    # the small workload's initial graph
    (777, 3, 5, 4, 2),        # d padded 3 -> 16, n not a multiple of either tile
    (600, 128, 10, 6, 3),
    (700, 96, 20, 8, 4),      # k = 20 (32-entry row lists); d 96 -> 128-wide BF16 rows
    (129, 64, 32, 3, 5),      # k = 32, the largest; one row past a 128-row tile
    (128, 32, 8, 3, 8),       # exactly one 128-row tile
    (300, 40, 31, 5, 10),     # d padded 40 -> 64; k = 31
    (33, 256, 32, 2, 6),      # n = k + 1, the smallest graph; d = 256, the largest
    (65, 100, 1, 2, 7),       # k = 1; d = 100 padded to 128
]


@pytest.mark.parametrize("path", ["cuda_cores", "tensor_cores"])
@pytest.mark.parametrize("n,d,k,comps,seed", EXACT_CASES)
def test_exact_graph_matches_oracle(knn, path, n, d, k, comps, seed):
    if path == "tensor_cores" and not tc_capable(n, d):
        pytest.skip("the tensor-core path needs padded d <= 128 and n >= 128")
    X = Mixture(d=d, components=comps, half_width=10.0, sigma=1.0, seed=seed).sample(n, seed + 100)
    ids, sims = gpu_exact(knn, X, k, path)
    o_ids, o_sims, margin = oracle.exact_knn(X, k)
    flagged = check_rows(ids, sims, o_ids, o_sims, margin, exact_tol(d))
    assert flagged <= n // 2   # k boundaries per row can each be a near tie


@pytest.mark.parametrize("path", ["cuda_cores", "tensor_cores"])
def test_exact_graph_duplicates_tie_to_lower_id(knn, path):
    X = Mixture(d=16, components=3, half_width=5.0, sigma=1.0, seed=9).sample(200, 1)
    X[50] = X[10]
    X[120] = X[10]
    ids, sims = gpu_exact(knn, X, 4, path)
    assert list(ids[10][:2]) == [50, 120] and sims[10][0] == 1.0
    assert list(ids[120][:2]) == [10, 50]


@pytest.mark.parametrize("n,d,k", [(500, 64, 10), (5000, 24, 20)])
def test_exact_tensor_cores_settle_unscreenable_rows(knn, n, d, k):
    """Points far from the origin (norms ~1e4 against distances ~1) make the
    screening error bound exceed every row's gap, so every row must go to the
    FP32 pass over all columns (split in column segments, merged per row);
    the lists stay exact."""
    X = Mixture(d=d, components=4, half_width=3.0, sigma=1.0, seed=12).sample(n, 3)
    X = (X + np.float32(2000.0)).astype(np.float32)
    ids, sims = gpu_exact(knn, X, k, "tensor_cores")
    info = knn.knn_exact_last_info()
    assert info["rows_redone"] == n
    rows = np.arange(n) if n <= 1000 else np.random.default_rng(2).choice(n, 200, replace=False)
    o_ids, o_sims, margin = oracle.exact_knn(X, k, rows=rows)
    # FP32 differences of coordinates near 2000 are exact (Sterbenz), so the
    # kernels' tolerance still applies
    check_rows(ids[rows], sims[rows], o_ids, o_sims, margin, exact_tol(d))


def test_exact_tensor_cores_refuse_what_they_cannot_do(knn):
    import torch
    X = cuda_tensor(Mixture(d=200, components=2, half_width=3.0, sigma=1.0, seed=1).sample(300, 1))
    ids = torch.empty((300, 5), dtype=torch.int64, device="cuda")
    knn.knn_exact_set_path("tensor_cores")
    try:
        with pytest.raises(knn.KnnError) as e:
            knn.knn_exact_graph(X, 5, ids)
        assert e.value.status == knn.KNN_ERR_UNSUPPORTED
    finally:
        knn.knn_exact_set_path("auto")


@pytest.mark.parametrize("n,d,k,seed", [(20_000, 128, 10, 13), (9_000, 16, 20, 14)])
def test_exact_tensor_cores_split_last_wave(knn, n, d, k, seed):
    """The row blocks of the last, partly filled wave of CTAs are screened in
    column parts and their lists merged per row: every one of the last 1,024
    rows (where those blocks lie) and 64 others against the oracle."""
    X = Mixture(d=d, components=30, half_width=10.0, sigma=1.0, seed=seed).sample(n, 4)
    ids, sims = gpu_exact(knn, X, k, "tensor_cores")
    assert knn.knn_exact_last_info()["rows_redone"] <= n // 100
    rng = np.random.default_rng(seed)
    rows = np.concatenate([rng.choice(n - 1024, 64, replace=False), np.arange(n - 1024, n)])
    o_ids, o_sims, margin = oracle.exact_knn(X, k, rows=rows)
    check_rows(ids[rows], sims[rows], o_ids, o_sims, margin, exact_tol(d))


def test_exact_graph_full_size_sampled_rows(knn):
    """The 100,000-point, d = 128 initial graph: 64 sampled rows against the
    oracle, and the list invariants on every row."""
    X = PLAIN_D128.initial()
    k = PLAIN_D128.k
    ids, sims = gpu_exact(knn, X, k)
    info = knn.knn_exact_last_info()
    assert info["path"] == "tensor_cores"
    assert info["rows_redone"] <= X.shape[0] // 100   # the screening settles almost every row
    # 48 rows anywhere and 16 of the last 2,048, where the last wave's row
    # blocks are screened in column parts
    rng = np.random.default_rng(5)
    rows = np.concatenate([rng.choice(X.shape[0] - 2048, 48, replace=False),
                           X.shape[0] - 2048 + rng.choice(2048, 16, replace=False)])
    o_ids, o_sims, margin = oracle.exact_knn(X, k, rows=rows)
    check_rows(ids[rows], sims[rows], o_ids, o_sims, margin, exact_tol(128))
    n = X.shape[0]
    assert ids.min() >= 0 and ids.max() < n
    assert not np.any(ids == np.arange(n)[:, None])
    srt = np.sort(ids, axis=1)
    assert not np.any(srt[:, 1:] == srt[:, :-1])
    assert np.all(np.diff(sims, axis=1) <= 0)


def test_exact_tensor_cores_wait_timeouts_are_detected_and_harmless(knn):
    """Failure detection without a fault: with a zero wait limit the
    pipeline roles give up on each other, the wait errors are reported, and
    the FP32 pass recomputes the affected rows, so the lists stay exact."""
    X = Mixture(d=64, components=6, half_width=10.0, sigma=1.0, seed=21).sample(1500, 2)
    knn.knn_exact_set_wait_limit(0)
    try:
        import torch
        out = torch.empty((1500, 10), dtype=torch.int64, device="cuda")
        osims = torch.empty((1500, 10), dtype=torch.float32, device="cuda")
        knn.knn_exact_set_path("tensor_cores")
        knn.knn_exact_graph(cuda_tensor(X), 10, out, osims)
        torch.cuda.synchronize()
        info = knn.knn_exact_last_info()
    finally:
        knn.knn_exact_set_wait_limit(-1)
        knn.knn_exact_set_path("auto")
    assert info["path"] == "tensor_cores" and info["wait_errors"] != 0 and info["rows_redone"] > 0
    o_ids, o_sims, margin = oracle.exact_knn(X, 10)
    check_rows(out.cpu().numpy(), osims.cpu().numpy(), o_ids, o_sims, margin, exact_tol(64))
    ids, _ = gpu_exact(knn, X, 10, "tensor_cores")   # the default limit again: no errors
    assert knn.knn_exact_last_info()["wait_errors"] == 0
