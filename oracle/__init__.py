"""FP64 CPU oracle for the online k-nn graph method (Debatty, Michiardi, Mees,
"Fast Online k-nn Graph Building", KDD'16).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package.  The product (the CUDA library
and its Python binding) never imports, links or runs anything here, and this
package never touches the product: the two share no code.  The arithmetic
lives in ``knn_oracle.c`` (plain C, FP64); this module compiles it with gcc and
marshals numpy arrays in and out.

Every function cites the passage of the paper it follows:

* :func:`exact_knn`     brute-force exact k-nn graph (Sec. 2.1; Sec. 8.5).
* :func:`search`        iGNNS (Sec. 3).
* :func:`rescore`       exact re-score of screening candidates.
* :func:`update`        Update (Algorithm 2).
* :func:`insert_stream` sequential online build (Algorithm 1).
* :func:`partitioned_search`, :func:`partitioned_search_labels`  distributed
  search (Sec. 5, Algorithm 3).
* :func:`kmedoids` and its steps  balanced k-medoids (Sec. 6, Algorithm 4).
* :func:`nearest_medoid`, :func:`medoid_recompute_sizes`,
  :func:`distributed_insert_stream`  distributed online build (Sec. 7,
  Algorithm 5; the recompute interval of Sec. 8.5).
* :func:`correct_edges`, :func:`quality_q`  graph quality (Sec. 8.5).
* :func:`quantize_bf16`, :func:`quantize_e4m3`  screening storage codes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libknn_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE arithmetic, no contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class SearchStats(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int64), ("budget", ctypes.c_int64),
                ("restarts", ctypes.c_int64), ("discarded", ctypes.c_int64),
                ("moves", ctypes.c_int64), ("draws", ctypes.c_int64),
                ("min_margin", ctypes.c_double)]


class UpdateStats(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int64), ("literal_evals", ctypes.c_int64),
                ("offers_taken", ctypes.c_int64), ("min_margin", ctypes.c_double)]


class InsertStats(ctypes.Structure):
    _fields_ = [("search_evals", ctypes.c_int64), ("update_evals", ctypes.c_int64),
                ("update_literal_evals", ctypes.c_int64),
                ("search_margin", ctypes.c_double), ("update_margin", ctypes.c_double)]


_P = ctypes.c_void_p
_I32, _I64, _U64, _F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "orc_similarity": (_F64, [_P, _P, _I32]),
                "orc_splitmix64_output": (_U64, [_U64, _U64]),
                "orc_search_key": (_U64, [_U64, _U64]),
                "orc_draw": (_I64, [_U64, _U64, _I64]),
                "orc_exact_knn": (None, [_P, _I64, _I32, _I32, _P, _I64, _P, _P, _P, _P]),
                "orc_search": (_I32, [_P, _I64, _I32, _P, _I32, _P, _P, _I32, _F64, _F64,
                                      _U64, _U64, _P, _I64, _P, _P, _P]),
                "orc_search_climb": (_I32, [_P, _I64, _I32, _P, _I32, _P, _P, _I32, _F64, _F64,
                                            _U64, _U64, _P, _I64, _I32, _P, _P, _P]),
                "orc_kmedoids_init": (None, [_I64, _I32, _U64, _P]),
                "orc_kmedoids_assign": (None, [_P, _I64, _I32, _P, _I32, _F64, _I32, _P, _P]),
                "orc_kmedoids_medoid": (_I64, [_P, _I32, _P, _I64, _P]),
                "orc_kmedoids": (None, [_P, _I64, _I32, _I32, _F64, _I32, _I32, _U64, _P, _P, _P]),
                "orc_rescore": (_I32, [_P, _I32, _P, _P, _I32, _I32, _P, _P, _P]),
                "orc_update": (None, [_P, _I64, _I32, _P, _P, _I32, _P, _I64, _P, _P, _I32,
                                      _I32, _I32, _P]),
                "orc_insert_stream": (None, [_P, _I64, _I64, _I32, _P, _P, _I32, _P, _F64,
                                             _F64, _I32, _U64, _P]),
                "orc_correct_edges": (_I64, [_P, _P, _I64, _I32]),
                "orc_quality_q": (_F64, [_I64, _I64, _I64, _I32]),
                "orc_bf16_code": (ctypes.c_uint16, [ctypes.c_float]),
                "orc_bf16_value": (ctypes.c_float, [ctypes.c_uint16]),
                "orc_e4m3_code": (ctypes.c_uint8, [ctypes.c_float]),
                "orc_e4m3_value": (ctypes.c_float, [ctypes.c_uint8]),
                "orc_quantize_bf16": (None, [_P, _I64, _P, _P]),
                "orc_quantize_e4m3": (None, [_P, _I64, _I32, _P, _P, _P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _removed(removed, n):
    if removed is None:
        return None
    r = np.ascontiguousarray(removed, dtype=np.uint8)
    assert r.shape[0] >= n
    return r


# --------------------------------------------------------------------------
# similarity and the restart generator
# --------------------------------------------------------------------------

def similarity(a, b) -> float:
    """sim(a, b) = 1/(1 + ||a - b||_2) in FP64 (the synthetic data's L2, Sec. 8.1)."""
    a, b = _f32(a), _f32(b)
    return _load().orc_similarity(_ptr(a), _ptr(b), a.shape[-1])


def splitmix64_output(seed: int, j: int) -> int:
    """Output j (0-based) of SplitMix64 seeded with `seed` (Steele et al. 2014)."""
    return _load().orc_splitmix64_output(seed, j)


def search_key(seed: int, stream: int) -> int:
    return _load().orc_search_key(seed, stream)


def draw(key: int, j: int, n: int) -> int:
    """Node picked by restart draw j: floor(x_j * n / 2^64)."""
    return _load().orc_draw(key, j, n)


# --------------------------------------------------------------------------
# exact graph
# --------------------------------------------------------------------------

def exact_knn(X, k: int, rows=None, removed=None):
    """Brute-force exact k-nn graph (Sec. 2.1): for every row u, the k nodes
    v != u of highest similarity, ties to the lower id.

    Returns (ids int64 [r, k], sims float64 [r, k], margin float64 [r]).
    """
    X = _f32(X)
    n, d = X.shape
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    r = n if rows_a is None else rows_a.shape[0]
    ids = np.empty((r, k), np.int64)
    sims = np.empty((r, k), np.float64)
    margin = np.empty(r, np.float64)
    _load().orc_exact_knn(_ptr(X), n, d, k, _ptr(rows_a), r, _ptr(_removed(removed, n)),
                          _ptr(ids), _ptr(sims), _ptr(margin))
    return ids, sims, margin


# --------------------------------------------------------------------------
# iGNNS, re-score, Update, sequential online build
# --------------------------------------------------------------------------

@dataclass
class SearchResult:
    ids: np.ndarray
    sims: np.ndarray
    evals: int
    budget: int
    restarts: int
    discarded: int
    moves: int
    draws: int
    margin: float


CLIMBS = {"eager": 0, "best": 1}


def search(X, nbr_ids, q, k_out: int, speedup: float, expansion: float,
           seed: int, stream: int, n: int | None = None, removed=None,
           draws=None, climb: str = "eager") -> SearchResult:
    """iGNNS (Sec. 3) over the first n rows of X with adjacency nbr_ids [n, k].
    climb="best" is the GNNS climb the paper compares against (every
    unvisited neighbour evaluated, move to the most similar); use it with
    expansion=inf for GNNS itself."""
    X = _f32(X)
    d = X.shape[1]
    n = X.shape[0] if n is None else n
    nbr = np.ascontiguousarray(nbr_ids, dtype=np.int64)
    k = nbr.shape[1]
    q = _f32(q)
    ids = np.empty(k_out, np.int64)
    sims = np.empty(k_out, np.float64)
    st = SearchStats()
    dr = None if draws is None else np.ascontiguousarray(draws, dtype=np.int64)
    _load().orc_search_climb(_ptr(X), n, d, _ptr(nbr), k, _ptr(_removed(removed, n)), _ptr(q),
                             k_out, float(speedup), float(expansion), seed, stream,
                             _ptr(dr), 0 if dr is None else dr.shape[0], CLIMBS[climb],
                             _ptr(ids), _ptr(sims), ctypes.byref(st))
    return SearchResult(ids, sims, st.evals, st.budget, st.restarts, st.discarded,
                        st.moves, st.draws, st.min_margin)


# --------------------------------------------------------------------------
# balanced k-medoids (Sec. 6, Algorithm 4)
# --------------------------------------------------------------------------

def kmedoids_init(n: int, p: int, seed: int) -> np.ndarray:
    """p distinct initial medoids drawn with the restart generator."""
    out = np.empty(p, np.int64)
    _load().orc_kmedoids_init(n, p, seed, _ptr(out))
    return out


def kmedoids_assign(X, medoids, imbalance: float, chunks: int):
    """Assign step with the capacity penalty w(t, m): (labels int32 [n],
    margins float64 [n])."""
    X = _f32(X)
    n, d = X.shape
    med = np.ascontiguousarray(medoids, dtype=np.int64)
    labels = np.empty(n, np.int32)
    margins = np.empty(n, np.float64)
    _load().orc_kmedoids_assign(_ptr(X), n, d, _ptr(med), med.shape[0], float(imbalance), chunks,
                                _ptr(labels), _ptr(margins))
    return labels, margins


def kmedoids_medoid(X, members):
    """Update step of one cluster: (medoid id, margin)."""
    X = _f32(X)
    mem = np.ascontiguousarray(members, dtype=np.int64)
    g = ctypes.c_double()
    m = _load().orc_kmedoids_medoid(_ptr(X), X.shape[1], _ptr(mem), mem.shape[0], ctypes.byref(g))
    return int(m), g.value


def kmedoids(X, p: int, imbalance: float, chunks: int, iters: int, seed: int):
    """Algorithm 4: (labels int32 [n], medoids int64 [p], smallest margin)."""
    X = _f32(X)
    n, d = X.shape
    labels = np.empty(n, np.int32)
    med = np.empty(p, np.int64)
    g = ctypes.c_double()
    _load().orc_kmedoids(_ptr(X), n, d, p, float(imbalance), chunks, iters, seed, _ptr(labels),
                         _ptr(med), ctypes.byref(g))
    return labels, med, g.value


PART_STREAM_STEP = 1 << 56


def partitioned_search(X, nbr_ids, q, k_out: int, part_offsets, speedup: float, expansion: float,
                       seed: int, stream: int, removed=None, climb: str = "eager"):
    """Distributed search (Sec. 5, Algorithm 3) with contiguous partitions:
    partition j (nodes part_offsets[j] .. part_offsets[j+1]-1) is searched on
    its own subgraph -- its rows, its lists with the entries that leave it
    dropped -- with budget max(1, floor(size / speedup)) and restart stream
    stream + j * 2^56; the k_out most similar of all candidates are kept.
    Returns (ids, sims, summed SearchResult counters, margin)."""
    X = _f32(X)
    nbr = np.ascontiguousarray(nbr_ids, dtype=np.int64)
    rem = None if removed is None else np.asarray(removed, dtype=np.uint8)
    ids_all, sims_all = [], []
    tot = dict(evals=0, restarts=0, discarded=0, moves=0, draws=0)
    margin = math.inf
    for j in range(len(part_offsets) - 1):
        lo, hi = int(part_offsets[j]), int(part_offsets[j + 1])
        if hi == lo:
            continue
        sub = nbr[lo:hi].copy()
        inside = (sub >= lo) & (sub < hi)
        sub = np.where(inside, sub - lo, -1)
        r = search(X[lo:hi], sub, q, k_out, speedup, expansion, seed,
                   (stream + j * PART_STREAM_STEP) % (1 << 64), n=hi - lo,
                   removed=None if rem is None else rem[lo:hi], climb=climb)
        for key in tot:
            tot[key] += getattr(r, key)
        margin = min(margin, r.margin)
        ok = r.ids >= 0
        ids_all.append(r.ids[ok] + lo)
        sims_all.append(r.sims[ok])
    ids = np.concatenate(ids_all) if ids_all else np.empty(0, np.int64)
    sims = np.concatenate(sims_all) if sims_all else np.empty(0)
    order = np.lexsort((ids, -sims))          # similarity descending, then id
    ids, sims = ids[order], sims[order]
    if len(sims) > k_out:                     # the boundary of the kept set
        a, b = sims[k_out - 1], sims[k_out]
        if a != b:
            margin = min(margin, abs(a - b) / max(abs(a), abs(b)))
    out_ids = np.full(k_out, -1, np.int64)
    out_sims = np.full(k_out, -np.inf)
    kk = min(k_out, len(ids))
    out_ids[:kk], out_sims[:kk] = ids[:kk], sims[:kk]
    return out_ids, out_sims, tot, margin


def partitioned_search_labels(X, nbr_ids, q, k_out: int, labels, parts: int, speedup: float,
                              expansion: float, seed: int, stream: int, climb: str = "eager"):
    """Distributed search (Sec. 5, Algorithm 3) over partitions given by a
    label per node: partition j, its nodes in id order, is searched on its own
    subgraph -- its rows, its lists with the entries that leave it dropped --
    with budget max(1, floor(size / speedup)) and restart stream
    stream + j * 2^56, whose draws index its nodes in id order; of all the
    partitions' results the k_out most similar are kept, ties to the lower
    id.  Returns (ids, sims, summed counters, margin) as partitioned_search."""
    X = _f32(X)
    labels = np.asarray(labels)
    n = labels.shape[0]
    nbr = np.ascontiguousarray(nbr_ids[:n], dtype=np.int64)
    ids_all, sims_all = [], []
    tot = dict(evals=0, restarts=0, discarded=0, moves=0, draws=0)
    margin = math.inf
    for j in range(parts):
        members = np.flatnonzero(labels == j)
        if members.size == 0:
            continue
        local = np.full(n, -1, np.int64)
        local[members] = np.arange(members.size)
        lists = nbr[members]
        inside = (lists >= 0) & (lists < n)
        lists = np.where(inside, local[np.where(inside, lists, 0)], -1)
        r = search(X[members], lists, q, k_out, speedup, expansion, seed,
                   (stream + j * PART_STREAM_STEP) % (1 << 64), n=members.size, climb=climb)
        for key in tot:
            tot[key] += getattr(r, key)
        margin = min(margin, r.margin)
        ok = r.ids >= 0
        ids_all.append(members[r.ids[ok]])
        sims_all.append(r.sims[ok])
    ids = np.concatenate(ids_all) if ids_all else np.empty(0, np.int64)
    sims = np.concatenate(sims_all) if sims_all else np.empty(0)
    order = np.lexsort((ids, -sims))
    ids, sims = ids[order], sims[order]
    if len(sims) > k_out:
        a, b = sims[k_out - 1], sims[k_out]
        if a != b:
            margin = min(margin, abs(a - b) / max(abs(a), abs(b)))
    out_ids = np.full(k_out, -1, np.int64)
    out_sims = np.full(k_out, -np.inf)
    kk = min(k_out, len(ids))
    out_ids[:kk], out_sims[:kk] = ids[:kk], sims[:kk]
    return out_ids, out_sims, tot, margin


def nearest_medoid(X, rows, medoids):
    """NearestMedoid of Algorithm 5: for each row the position of the most
    similar medoid, sim = 1/(1 + L2) in FP64, ties to the lower position.
    Returns (labels int32, margins float64: the relative gap between the best
    and the second-best similarity, inf with one medoid)."""
    X = _f32(X)
    R = X[np.asarray(rows, dtype=np.int64)].astype(np.float64)
    M = X[np.asarray(medoids, dtype=np.int64)].astype(np.float64)
    sims = 1.0 / (1.0 + np.sqrt(((R[:, None, :] - M[None, :, :]) ** 2).sum(-1)))
    labels = np.argmax(sims, axis=1).astype(np.int32)      # the first maximum: the lower position
    if M.shape[0] == 1:
        return labels, np.full(R.shape[0], np.inf)
    top2 = -np.sort(-sims, axis=1)[:, :2]
    margins = np.abs(top2[:, 0] - top2[:, 1]) / np.maximum(np.abs(top2[:, 0]), np.abs(top2[:, 1]))
    return labels, margins


def medoid_recompute_sizes(n_last: int, n_end: int, interval: float, batch: int = 1):
    """Graph sizes at which the medoids are recomputed (Sec. 8.5, "Interval
    between recomputing medoids"): growing by `batch` nodes at a time from
    n_last to n_end, after every step that leaves the graph at least
    interval * (its size at the last recompute) nodes larger than then."""
    out, n = [], n_last
    if interval <= 0:
        return out
    while n < n_end:
        n = min(n + batch, n_end)
        if n - n_last >= interval * n_last:
            out.append(n)
            n_last = n
    return out


def distributed_insert_stream(G: "Graph", Xnew, labels, medoids, speedup: float, expansion: float,
                              depth: int, seed: int, interval: float, n_last: int | None = None,
                              climb: str = "eager") -> dict:
    """Distributed online build (Sec. 7, Algorithm 5), one new point at a
    time on the sequential graph G: the distributed search over the label
    partitions (restart stream = the new id), Update (Algorithm 2) over the
    whole graph, the new node given to the partition of its nearest medoid;
    then, when the graph has grown by interval * n_last nodes since the last
    recompute, every non-empty partition takes the member with the smallest
    sum of Euclidean distances to the others as its medoid (Algorithm 4's
    update step).  labels (capacity-long int32) and medoids (int64) are
    updated in place.  Returns per-insert margins and the recompute count."""
    Xnew = _f32(Xnew)
    parts = len(medoids)
    n_last = G.n if n_last is None else n_last
    stats = dict(search_margin=[], update_margin=[], assign_margin=[], recompute_margin=[],
                 search_evals=[], update_evals=[], recomputes=0)
    for x in Xnew:
        i = G.n
        G.X[i] = x
        ids, sims, ctr, sm = partitioned_search_labels(G.X[:i], G.ids[:i], G.X[i], G.k, labels[:i], parts,
                                                       speedup, expansion, seed, i, climb=climb)
        G.ids[i], G.sims[i] = ids, sims
        u = update(G.X, i + 1, G.ids, G.sims, i, ids, sims, depth, removed=G.removed[: i + 1])
        lab, am = nearest_medoid(G.X, [i], medoids)
        labels[i] = lab[0]
        G.n = i + 1
        stats["search_margin"].append(sm)
        stats["update_margin"].append(u.min_margin)
        stats["assign_margin"].append(am[0])
        stats["search_evals"].append(ctr["evals"])
        stats["update_evals"].append(u.evals)
        if interval > 0 and G.n - n_last >= interval * n_last:
            rm = math.inf
            for j in range(parts):
                members = np.flatnonzero(labels[: G.n] == j)
                if members.size:
                    medoids[j], gap = kmedoids_medoid(G.X[: G.n], members)
                    rm = min(rm, gap)
            stats["recompute_margin"].append(rm)
            stats["recomputes"] += 1
            n_last = G.n
    stats["n_last"] = n_last
    return stats


def rescore(X, q, cand_ids, k_out: int):
    """Exact similarities of q to the candidates; keep the k_out best."""
    X = _f32(X)
    q = _f32(q)
    c = np.ascontiguousarray(cand_ids, dtype=np.int64)
    ids = np.empty(k_out, np.int64)
    sims = np.empty(k_out, np.float64)
    margin = ctypes.c_double()
    _load().orc_rescore(_ptr(X), X.shape[1], _ptr(q), _ptr(c), c.shape[0], k_out,
                        _ptr(ids), _ptr(sims), ctypes.byref(margin))
    return ids, sims, margin.value


def update(X, n_total: int, nbr_ids: np.ndarray, nbr_sims: np.ndarray, new_id: int,
           L_ids, L_sims, depth: int, removed=None, full: bool = False) -> UpdateStats:
    """Update (Algorithm 2) in place on nbr_ids (int64) / nbr_sims (float64)."""
    X = _f32(X)
    assert nbr_ids.dtype == np.int64 and nbr_sims.dtype == np.float64
    assert nbr_ids.flags["C_CONTIGUOUS"] and nbr_sims.flags["C_CONTIGUOUS"]
    k = nbr_ids.shape[1]
    Li = np.ascontiguousarray(L_ids, dtype=np.int64)
    Ls = np.ascontiguousarray(L_sims, dtype=np.float64)
    st = UpdateStats()
    _load().orc_update(_ptr(X), n_total, X.shape[1], _ptr(nbr_ids), _ptr(nbr_sims), k,
                       _ptr(_removed(removed, n_total)), new_id, _ptr(Li), _ptr(Ls),
                       Li.shape[0], depth, int(full), ctypes.byref(st))
    return st


class Graph:
    """Sequential online graph (Algorithm 1) held in numpy arrays."""

    def __init__(self, d: int, k: int, capacity: int):
        self.d, self.k, self.capacity = d, k, capacity
        self.X = np.zeros((capacity, d), np.float32)
        self.ids = np.full((capacity, k), -1, np.int64)
        self.sims = np.full((capacity, k), -np.inf, np.float64)
        self.removed = np.zeros(capacity, np.uint8)
        self.n = 0

    @classmethod
    def exact(cls, X0, k: int, capacity: int | None = None) -> "Graph":
        """Initial graph: the brute-force exact graph of X0 (Sec. 8.5)."""
        X0 = _f32(X0)
        g = cls(X0.shape[1], k, capacity or X0.shape[0])
        g.X[: X0.shape[0]] = X0
        ids, sims, _ = exact_knn(X0, k)
        g.ids[: X0.shape[0]] = ids
        g.sims[: X0.shape[0]] = sims
        g.n = X0.shape[0]
        return g

    def insert_stream(self, Xnew, speedup: float, expansion: float, depth: int,
                      seed: int) -> np.ndarray:
        """Algorithm 1 for every row of Xnew in order; returns per-insert stats
        as a structured array (search_evals, update_evals, ..., margins)."""
        Xnew = _f32(Xnew)
        m = Xnew.shape[0]
        assert self.n + m <= self.capacity
        self.X[self.n: self.n + m] = Xnew
        stats = (InsertStats * m)()
        _load().orc_insert_stream(_ptr(self.X), self.n, m, self.d, _ptr(self.ids),
                                  _ptr(self.sims), self.k, _ptr(self.removed),
                                  float(speedup), float(expansion), depth, seed, stats)
        self.n += m
        return np.array([(s.search_evals, s.update_evals, s.update_literal_evals,
                          s.search_margin, s.update_margin) for s in stats],
                        dtype=[("search_evals", "i8"), ("update_evals", "i8"),
                               ("update_literal_evals", "i8"), ("search_margin", "f8"),
                               ("update_margin", "f8")])

    def search(self, q, k_out, speedup, expansion, seed, stream, climb="eager") -> SearchResult:
        return search(self.X, self.ids[: self.n], q, k_out, speedup, expansion, seed,
                      stream, n=self.n, removed=self.removed, climb=climb)


# --------------------------------------------------------------------------
# graph quality (Sec. 8.5)
# --------------------------------------------------------------------------

def correct_edges(ids_online, ids_exact) -> int:
    """e_c: directed edges u->v present in both graphs."""
    a = np.ascontiguousarray(ids_online, dtype=np.int64)
    b = np.ascontiguousarray(ids_exact, dtype=np.int64)
    assert a.shape == b.shape
    return _load().orc_correct_edges(_ptr(a), _ptr(b), a.shape[0], a.shape[1])


def quality_q(e_c: int, n: int, n_a: int, k: int) -> float:
    """Q = (e_c - e_u)/e_m (Sec. 8.5)."""
    return _load().orc_quality_q(e_c, n, n_a, k)


# --------------------------------------------------------------------------
# screening storage codes
# --------------------------------------------------------------------------

def quantize_bf16(X):
    """BF16 codes (uint16) and their values (float32) of every element."""
    X = _f32(X)
    codes = np.empty(X.shape, np.uint16)
    deq = np.empty(X.shape, np.float32)
    _load().orc_quantize_bf16(_ptr(X), X.size, _ptr(codes), _ptr(deq))
    return codes, deq


def quantize_e4m3(X):
    """FP8-E4M3 codes with a per-row scale amax/448: (codes uint8 [n, d],
    scales float32 [n], dequantized float32 [n, d])."""
    X = _f32(X)
    n, d = X.shape
    codes = np.empty((n, d), np.uint8)
    scales = np.empty(n, np.float32)
    deq = np.empty((n, d), np.float32)
    _load().orc_quantize_e4m3(_ptr(X), n, d, _ptr(codes), _ptr(scales), _ptr(deq))
    return codes, scales, deq


def bf16_code(x: float) -> int:
    return _load().orc_bf16_code(x)


def e4m3_code(x: float) -> int:
    return _load().orc_e4m3_code(x)


def e4m3_value(c: int) -> float:
    return _load().orc_e4m3_value(c)
