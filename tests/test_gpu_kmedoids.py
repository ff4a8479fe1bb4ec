"""Balanced k-medoids (Sec. 6, Algorithm 4) on the GPU against the FP64
oracle: the initial medoids bit-exact; the assignment of every chunk
identical up to its first decision whose margin is within FP32 reach (one
flipped decision changes the later penalties, so the comparison of a chunk
stops there); the medoid update identical where its margin is safe; the
ordering a stable sort by (cluster, id)."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import U, cuda_tensor, padded
from paper_1602_06819_gb300.inputs import Mixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


def gpu_kmedoids(knn, X, p, imbalance, chunks, iters, seed, device=True):
    import torch
    n = X.shape[0]
    dev = "cuda" if device else "cpu"
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    med = torch.empty(p, dtype=torch.int64, device=dev)
    order = torch.empty(n, dtype=torch.int64, device=dev)
    offsets = torch.empty(p + 1, dtype=torch.int64, device=dev)
    Xin = cuda_tensor(X) if device else np.ascontiguousarray(X)
    knn.knn_balanced_kmedoids(Xin, p, imbalance, chunks, iters, seed, labels, med, order, offsets)
    torch.cuda.synchronize()
    return labels.cpu().numpy(), med.cpu().numpy(), order.cpu().numpy(), offsets.cpu().numpy()


def assign_tol(d, n, p, chunks, imbalance):
    """Relative margin below which an assign decision may flip in FP32: the
    squared distance (DP + 2 roundings), sqrt, 1 + ., the division, the
    product, and the weight w = 1 - count / capacity, whose relative error
    is about (count / capacity) / w + 1 roundings, at most capacity + 1 while
    w >= 1 / capacity."""
    cap = n * imbalance / (p * chunks)
    cap = 1.0 if math.isinf(cap) else cap
    return 4.0 * (padded(d) + 10 + 2.0 * cap) * U


def check_order(labels, order, offsets, p):
    n = labels.shape[0]
    assert sorted(order.tolist()) == list(range(n))
    assert offsets[0] == 0 and offsets[-1] == n
    assert np.array_equal(np.diff(offsets), np.bincount(labels, minlength=p))
    for m in range(p):
        seg = order[offsets[m]:offsets[m + 1]]
        assert np.all(labels[seg] == m) and np.all(np.diff(seg) > 0)


def compare_assign(labels, o_labels, o_margin, n, chunks, tol, sequential=True):
    """Labels equal up to each chunk's first ambiguous decision (without the
    penalty the decisions are independent: equal wherever unambiguous);
    returns the number of decisions compared."""
    if not sequential:
        safe = o_margin >= tol
        assert np.array_equal(labels[safe], o_labels[safe])
        return int(safe.sum())
    compared = 0
    for c in range(chunks):
        lo, hi = c * n // chunks, (c + 1) * n // chunks
        amb = np.flatnonzero(o_margin[lo:hi] < tol)
        stop = hi if amb.size == 0 else lo + int(amb[0])
        assert np.array_equal(labels[lo:stop], o_labels[lo:stop]), f"chunk {c}"
        compared += stop - lo
    return compared


@pytest.mark.parametrize("n,d,p,chunks,imbalance,seed", [
    (3000, 16, 16, 4, 1.1, 1),
    (2500, 3, 10, 1, 1.0, 2),       # d padded 3 -> 16; exact balance
    (4000, 96, 40, 8, 1.2, 3),
    (1000, 128, 1, 2, 1.1, 4),      # one cluster
    (1500, 64, 30, 3, math.inf, 5),  # no penalty: nearest medoid
    (700, 256, 64, 1, 1.05, 6),     # the widest rows
])
def test_assign_matches_oracle(knn, n, d, p, chunks, imbalance, seed):
    mix = Mixture(d=d, components=max(2, p // 2), half_width=8.0, sigma=1.0, seed=seed)
    X = mix.sample(n, seed + 10)
    labels, med, order, offsets = gpu_kmedoids(knn, X, p, imbalance, chunks, 0, seed)
    assert np.array_equal(med, oracle.kmedoids_init(n, p, seed))
    o_labels, o_margin = oracle.kmedoids_assign(X, med, imbalance, chunks)
    compared = compare_assign(labels, o_labels, o_margin, n, chunks, assign_tol(d, n, p, chunks, imbalance),
                              sequential=not math.isinf(imbalance))
    assert compared >= n // 4
    check_order(labels, order, offsets, p)
    if not math.isinf(imbalance):
        cap = n * imbalance / (p * chunks)
        for c in range(chunks):
            lo, hi = c * n // chunks, (c + 1) * n // chunks
            assert np.bincount(labels[lo:hi], minlength=p).max() <= math.ceil(cap) + (imbalance == 1.0)


@pytest.mark.parametrize("n,d,p,chunks,imb,mix_seed", [(1600, 8, 4, 2, 2.0, 10), (1000, 4, 5, 1, 2.0, 10)])
def test_update_and_iterations_match_oracle(knn, n, d, p, chunks, imb, mix_seed):
    """Two rounds of (assign, update) then a final assign, on well separated
    clusters whose decisions all have safe margins on the oracle's side (the
    update sums a cluster's distances in FP32: a relative error of about
    (cluster size) roundings)."""
    X = Mixture(d=d, components=p, half_width=30.0, sigma=1.0, seed=mix_seed).sample(n, 1)
    o_labels, o_med, o_min = oracle.kmedoids(X, p, imb, chunks, 2, seed=7)
    tol = max(assign_tol(d, n, p, chunks, imb), 4.0 * (np.bincount(o_labels).max() + padded(d)) * U)
    assert o_min > tol, "fixture must be unambiguous"
    labels, med, order, offsets = gpu_kmedoids(knn, X, p, imb, chunks, 2, 7)
    assert np.array_equal(med, o_med)
    assert np.array_equal(labels, o_labels)
    check_order(labels, order, offsets, p)


def test_host_buffers_and_bad_arguments(knn):
    X = Mixture(d=16, components=4, half_width=8.0, sigma=1.0, seed=2).sample(600, 1)
    a = gpu_kmedoids(knn, X, 6, 1.1, 2, 1, 9, device=False)
    b = gpu_kmedoids(knn, X, 6, 1.1, 2, 1, 9, device=True)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    with pytest.raises(knn.KnnError):
        knn.knn_balanced_kmedoids(cuda_tensor(X), 2000, 1.1, 1, 0, 1)      # p > 1024
    with pytest.raises(knn.KnnError):
        knn.knn_balanced_kmedoids(cuda_tensor(X), 6, 0.5, 1, 0, 1)         # imbalance < 1
    with pytest.raises(knn.KnnError):
        knn.knn_balanced_kmedoids(cuda_tensor(X[:4]), 6, 1.1, 1, 0, 1)     # n < p
