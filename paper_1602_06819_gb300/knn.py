"""ctypes binding of the C ABI in include/knn_graph.h.

The functions keep the C names (knn_graph_create, knn_graph_insert_batch,
...) and only marshal arguments: every step of the method runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU, contiguous) or numpy
arrays; CUDA tensors pass their device pointer, everything else its host
pointer, and the library stages host memory itself.  `stream` defaults to
torch's current CUDA stream.

Importing this module loads libknn_graph.so and raises if it is missing or
cannot be loaded: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB

KNN_OK = 0
KNN_ERR_INVALID_ARG = -1
KNN_ERR_OOM = -2
KNN_ERR_CAPACITY = -3
KNN_ERR_CUDA = -4
KNN_ERR_DEVICE_TIMEOUT = -5
KNN_ERR_NOT_FOUND = -6
KNN_ERR_UNSUPPORTED = -7

KNN_CLIMB_EAGER = 0
KNN_CLIMB_BEST = 1
CLIMBS = {"eager": KNN_CLIMB_EAGER, "best": KNN_CLIMB_BEST}

KNN_STORAGE_FP32 = 0
KNN_STORAGE_BF16 = 1
KNN_STORAGE_FP8_E4M3 = 2

NCOUNTERS = 8
COUNTER_NAMES = ("search_evals", "update_evals", "restarts", "discarded", "moves",
                 "adjacency_reads", "draws", "pad")

# Every symbol include/knn_graph.h declares.
EXPORTED = ("knn_graph_create", "knn_graph_restore", "knn_graph_insert_batch", "knn_graph_query_batch",
            "knn_graph_query_ids", "knn_graph_query_partitioned", "knn_graph_query_partitioned_ids",
            "knn_graph_remove", "knn_graph_get_edges",
            "knn_graph_reserve",
            "knn_graph_set_partitions", "knn_graph_insert_distributed", "knn_graph_get_partitions",
            "knn_graph_last_counters",
            "knn_graph_set_timing", "knn_graph_last_timing", "knn_graph_set_search", "knn_graph_stats",
            "knn_graph_destroy", "knn_exact_graph", "knn_exact_set_path", "knn_exact_last_info",
            "knn_exact_set_wait_limit",
            "knn_balanced_kmedoids", "knn_server_create", "knn_server_submit", "knn_server_wait",
            "knn_server_get_stats", "knn_server_destroy", "knn_multi_create", "knn_multi_step",
            "knn_multi_set_launch", "knn_multi_set_order", "knn_multi_graph_size", "knn_multi_get_edges", "knn_multi_destroy",
            "knn_search_noalloc",
            "knn_last_error", "knn_version")

KNN_REQ_INSERT = 0
KNN_REQ_QUERY = 1

EXACT_PATHS = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}

PHASES = ("store", "search", "rescore", "cross", "offers", "merge")


class KnnParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("k", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("speedup", ctypes.c_double),
                ("expansion", ctypes.c_double), ("rescore_mult", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("capacity", ctypes.c_int64)]


class KnnStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n", "capacity", "removed", "inserts", "queries", "search_evals", "update_evals",
        "cross_evals", "rescore_evals", "restarts", "moves", "adjacency_reads", "offers",
        "device_bytes", "kernel_launches")]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class KnnExactInfo(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("wait_errors", ctypes.c_uint32), ("n", ctypes.c_int64),
                ("rows_redone", ctypes.c_int64)]


class KnnServerParams(ctypes.Structure):
    _fields_ = [("k_out", ctypes.c_int32), ("max_step_points", ctypes.c_int32),
                ("grow_headroom_bytes", ctypes.c_int64), ("query_parts", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("part_offsets", ctypes.c_void_p)]


class KnnRequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("m", ctypes.c_int64),
                ("epoch", ctypes.c_int64), ("step", ctypes.c_int64), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class KnnServerStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("requests", ctypes.c_int64), ("points", ctypes.c_int64),
                ("inserts", ctypes.c_int64), ("queries", ctypes.c_int64), ("epoch", ctypes.c_int64),
                ("max_queue", ctypes.c_int64), ("busy_ms", ctypes.c_double), ("grows", ctypes.c_int64),
                ("capacity", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class KnnError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _load_library() -> ctypes.CDLL:
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sigs = {
        "knn_graph_create": (I32, [ctypes.POINTER(KnnParams), P, I64, P, ctypes.POINTER(P)]),
        "knn_graph_restore": (I32, [ctypes.POINTER(KnnParams), P, I64, P, P, ctypes.POINTER(P)]),
        "knn_graph_insert_batch": (I32, [P, P, I64, P, P, P]),
        "knn_graph_query_batch": (I32, [P, P, I64, I32, U64, P, P, P]),
        "knn_graph_query_partitioned": (I32, [P, P, I64, I32, U64, P, I32, P, P, P]),
        "knn_graph_query_ids": (I32, [P, P, I64, I32, P, P, P, P]),
        "knn_graph_query_partitioned_ids": (I32, [P, P, I64, I32, P, P, I32, P, P, P]),
        "knn_graph_remove": (I32, [P, P, I64, P]),
        "knn_graph_reserve": (I32, [P, I64, I64, P]),
        "knn_graph_set_partitions": (I32, [P, P, P, I32, ctypes.c_double, P]),
        "knn_graph_insert_distributed": (I32, [P, P, I64, P, P, P]),
        "knn_graph_get_partitions": (I32, [P, P, P, P, P]),
        "knn_graph_get_edges": (I32, [P, P, P, I64, ctypes.POINTER(I64), P]),
        "knn_graph_last_counters": (I32, [P, P, I64, P]),
        "knn_graph_set_timing": (I32, [P, I32]),
        "knn_graph_last_timing": (I32, [P, ctypes.POINTER(ctypes.c_float), I32]),
        "knn_graph_stats": (I32, [P, ctypes.POINTER(KnnStats)]),
        "knn_graph_destroy": (None, [P]),
        "knn_exact_graph": (I32, [P, I64, I32, I32, P, P, P]),
        "knn_exact_set_path": (I32, [I32]),
        "knn_exact_set_wait_limit": (I32, [I64]),
        "knn_server_create": (I32, [P, ctypes.POINTER(KnnServerParams), ctypes.POINTER(P)]),
        "knn_server_submit": (I32, [P, I32, P, I64, ctypes.POINTER(U64)]),
        "knn_server_wait": (I32, [P, U64, P, P, ctypes.POINTER(KnnRequestInfo)]),
        "knn_server_get_stats": (I32, [P, ctypes.POINTER(KnnServerStats)]),
        "knn_server_destroy": (None, [P]),
        "knn_multi_create": (I32, [ctypes.POINTER(KnnParams), I32, P, P, P, I32, P, ctypes.POINTER(P)]),
        "knn_multi_step": (I32, [P, P, P, P, P, I64, P, P, P]),
        "knn_multi_set_launch": (I32, [P, I32]),
        "knn_multi_set_order": (I32, [P, I32]),
        "knn_multi_graph_size": (I32, [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "knn_multi_get_edges": (I32, [P, I32, P, P]),
        "knn_multi_destroy": (None, [P]),
        "knn_balanced_kmedoids": (I32, [P, I64, I32, I32, ctypes.c_double, I32, I32, U64, P, P, P, P, P]),
        "knn_graph_set_search": (I32, [P, ctypes.c_double, ctypes.c_double, I32]),
        "knn_exact_last_info": (I32, [ctypes.POINTER(KnnExactInfo)]),
        "knn_search_noalloc": (I32, [P, I64, I32, P, I32, P, I64, I32, ctypes.c_double,
                                     ctypes.c_double, U64, U64, P, P, P]),
        "knn_last_error": (ctypes.c_char_p, []),
        "knn_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load_library()


def _check(status: int, where: str) -> None:
    if status != KNN_OK:
        raise KnnError(status, where, lib.knn_last_error().decode())


def _ptr(a) -> int | None:
    """Data pointer of a torch tensor or numpy array (None stays None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr()


def _stream(stream) -> int | None:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check_dtype(a, kind: str, name: str):
    if a is None:
        return
    dt = str(a.dtype)
    if kind not in dt:
        raise TypeError(f"{name} must be {kind}, got {dt}")


# --------------------------------------------------------------------------
# the C calls, same names
# --------------------------------------------------------------------------

def knn_graph_create(params: KnnParams, init_vecs, stream=None) -> ctypes.c_void_p:
    _check_dtype(init_vecs, "float32", "init_vecs")
    handle = ctypes.c_void_p()
    _check(lib.knn_graph_create(ctypes.byref(params), _ptr(init_vecs), init_vecs.shape[0],
                                _stream(stream), ctypes.byref(handle)), "knn_graph_create")
    return handle


def knn_graph_restore(params: KnnParams, vecs, nbr_ids, stream=None) -> ctypes.c_void_p:
    _check_dtype(vecs, "float32", "vecs")
    _check_dtype(nbr_ids, "int64", "nbr_ids")
    handle = ctypes.c_void_p()
    _check(lib.knn_graph_restore(ctypes.byref(params), _ptr(vecs), vecs.shape[0], _ptr(nbr_ids),
                                 _stream(stream), ctypes.byref(handle)), "knn_graph_restore")
    return handle


def knn_graph_insert_batch(g, vecs, out_ids=None, out_nbrs=None, stream=None) -> None:
    _check_dtype(vecs, "float32", "vecs")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_nbrs, "int64", "out_nbrs")
    _check(lib.knn_graph_insert_batch(g, _ptr(vecs), vecs.shape[0], _ptr(out_ids), _ptr(out_nbrs),
                                      _stream(stream)), "knn_graph_insert_batch")


def knn_graph_query_batch(g, vecs, k_out: int, query_id0: int, out_ids, out_sims=None,
                          stream=None) -> None:
    _check_dtype(vecs, "float32", "vecs")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_sims, "float32", "out_sims")
    _check(lib.knn_graph_query_batch(g, _ptr(vecs), vecs.shape[0], k_out, query_id0, _ptr(out_ids),
                                     _ptr(out_sims), _stream(stream)), "knn_graph_query_batch")


def knn_graph_query_ids(g, vecs, k_out: int, query_ids, out_ids, out_sims=None, stream=None) -> None:
    """Queries with their own restart streams 2^63 + query_ids[i] (uint64)."""
    _check_dtype(vecs, "float32", "vecs")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_sims, "float32", "out_sims")
    if str(query_ids.dtype) not in ("uint64", "torch.uint64", "int64", "torch.int64"):
        raise TypeError("query_ids must be 64-bit integers")
    _check(lib.knn_graph_query_ids(g, _ptr(vecs), vecs.shape[0], k_out, _ptr(query_ids), _ptr(out_ids),
                                   _ptr(out_sims), _stream(stream)), "knn_graph_query_ids")


def knn_graph_query_partitioned(g, vecs, k_out: int, query_id0: int, part_offsets, out_ids,
                                out_sims=None, stream=None) -> None:
    """Algorithm 3: search each partition (node ranges part_offsets[j] ..
    part_offsets[j+1]-1, int64 [parts + 1]) and keep the k_out best."""
    _check_dtype(vecs, "float32", "vecs")
    _check_dtype(part_offsets, "int64", "part_offsets")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_sims, "float32", "out_sims")
    _check(lib.knn_graph_query_partitioned(g, _ptr(vecs), vecs.shape[0], k_out, query_id0,
                                           _ptr(part_offsets), part_offsets.shape[0] - 1,
                                           _ptr(out_ids), _ptr(out_sims), _stream(stream)),
           "knn_graph_query_partitioned")


def knn_graph_query_partitioned_ids(g, vecs, k_out: int, query_ids, part_offsets, out_ids,
                                    out_sims=None, stream=None) -> None:
    """Algorithm 3 with one restart stream per query (2^63 + query_ids[i])."""
    _check_dtype(vecs, "float32", "vecs")
    _check_dtype(part_offsets, "int64", "part_offsets")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_sims, "float32", "out_sims")
    _check(lib.knn_graph_query_partitioned_ids(g, _ptr(vecs), vecs.shape[0], k_out, _ptr(query_ids),
                                               _ptr(part_offsets), part_offsets.shape[0] - 1,
                                               _ptr(out_ids), _ptr(out_sims), _stream(stream)),
           "knn_graph_query_partitioned_ids")


def knn_graph_set_partitions(g, labels, medoids, recompute_interval: float = 0.0, stream=None) -> None:
    """Algorithm 5's partitions: labels (int32 [n]) and medoids (int64 [parts])."""
    _check_dtype(labels, "int32", "labels")
    _check_dtype(medoids, "int64", "medoids")
    _check(lib.knn_graph_set_partitions(g, _ptr(labels), _ptr(medoids), medoids.shape[0], float(recompute_interval),
                                        _stream(stream)), "knn_graph_set_partitions")


def knn_graph_insert_distributed(g, vecs, out_ids=None, out_nbrs=None, stream=None) -> None:
    """Algorithm 5 for a batch: the distributed search, Update, nearest medoid."""
    _check_dtype(vecs, "float32", "vecs")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_nbrs, "int64", "out_nbrs")
    _check(lib.knn_graph_insert_distributed(g, _ptr(vecs), vecs.shape[0], _ptr(out_ids), _ptr(out_nbrs),
                                            _stream(stream)), "knn_graph_insert_distributed")


def knn_graph_get_partitions(g, labels=None, medoids=None, stream=None) -> int:
    """Fills labels (int32 [n]) and medoids (int64 [parts]); returns the
    number of medoid recomputes so far."""
    _check_dtype(labels, "int32", "labels")
    _check_dtype(medoids, "int64", "medoids")
    rec = ctypes.c_int64()
    _check(lib.knn_graph_get_partitions(g, _ptr(labels), _ptr(medoids), ctypes.addressof(rec), _stream(stream)),
           "knn_graph_get_partitions")
    return rec.value


def knn_graph_remove(g, ids, stream=None) -> None:
    _check_dtype(ids, "int64", "ids")
    _check(lib.knn_graph_remove(g, _ptr(ids), ids.shape[0], _stream(stream)), "knn_graph_remove")


def knn_graph_reserve(g, capacity: int, headroom_bytes: int = 0, stream=None) -> None:
    _check(lib.knn_graph_reserve(g, capacity, headroom_bytes, _stream(stream)), "knn_graph_reserve")


def knn_graph_get_edges(g, out_ids, out_sims=None, stream=None) -> int:
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_sims, "float32", "out_sims")
    n_out = ctypes.c_int64()
    _check(lib.knn_graph_get_edges(g, _ptr(out_ids), _ptr(out_sims), out_ids.shape[0],
                                   ctypes.byref(n_out), _stream(stream)), "knn_graph_get_edges")
    return n_out.value


def knn_graph_last_counters(g, out, stream=None) -> None:
    _check_dtype(out, "int64", "out")
    _check(lib.knn_graph_last_counters(g, _ptr(out), out.shape[0], _stream(stream)),
           "knn_graph_last_counters")


def knn_graph_set_search(handle, speedup: float, expansion: float, climb: str = "eager") -> None:
    """Search parameters of later inserts and queries; climb "eager" (iGNNS)
    or "best" (GNNS, with expansion=inf as the paper compares it)."""
    _check(lib.knn_graph_set_search(handle, float(speedup), float(expansion), CLIMBS[climb]),
           "knn_graph_set_search")


def knn_graph_set_timing(g, enable: bool) -> None:
    _check(lib.knn_graph_set_timing(g, int(bool(enable))), "knn_graph_set_timing")


def knn_graph_last_timing(g) -> dict:
    out = (ctypes.c_float * len(PHASES))()
    _check(lib.knn_graph_last_timing(g, out, len(PHASES)), "knn_graph_last_timing")
    return dict(zip(PHASES, list(out)))


def knn_graph_stats(g) -> dict:
    st = KnnStats()
    _check(lib.knn_graph_stats(g, ctypes.byref(st)), "knn_graph_stats")
    return st.as_dict()


def knn_graph_destroy(g) -> None:
    lib.knn_graph_destroy(g)


def knn_exact_graph(X, k: int, out_ids, out_sims=None, stream=None) -> None:
    _check_dtype(X, "float32", "X")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_sims, "float32", "out_sims")
    _check(lib.knn_exact_graph(_ptr(X), X.shape[0], X.shape[1], k, _ptr(out_ids), _ptr(out_sims),
                               _stream(stream)), "knn_exact_graph")


def knn_balanced_kmedoids(X, p: int, imbalance: float, chunks: int, iters: int, seed: int,
                          labels=None, medoids=None, order=None, offsets=None, stream=None) -> None:
    """Balanced k-medoids (Algorithm 4) of X [n, dim] float32; outputs
    labels [n] int32, medoids [p] int64, order [n] int64 (position -> point,
    clusters contiguous), offsets [p + 1] int64, each optional."""
    _check_dtype(X, "float32", "X")
    _check_dtype(labels, "int32", "labels")
    for name, arr in (("medoids", medoids), ("order", order), ("offsets", offsets)):
        _check_dtype(arr, "int64", name)
    _check(lib.knn_balanced_kmedoids(_ptr(X), X.shape[0], X.shape[1], p, float(imbalance), chunks,
                                     iters, seed, _ptr(labels), _ptr(medoids), _ptr(order),
                                     _ptr(offsets), _stream(stream)), "knn_balanced_kmedoids")


def knn_exact_set_path(path: str) -> None:
    """Process-wide choice of the exact-graph path: "auto", "cuda_cores" or "tensor_cores"."""
    _check(lib.knn_exact_set_path(EXACT_PATHS[path]), "knn_exact_set_path")


def knn_exact_set_wait_limit(ns: int) -> None:
    """Pipeline wait limit of the tensor-core build (ns < 0: default 2 s)."""
    _check(lib.knn_exact_set_wait_limit(int(ns)), "knn_exact_set_wait_limit")


def knn_exact_last_info() -> dict:
    """The calling thread's last exact build: path, n, rows redone by brute force, wait errors."""
    info = KnnExactInfo()
    _check(lib.knn_exact_last_info(ctypes.byref(info)), "knn_exact_last_info")
    names = {v: k for k, v in EXACT_PATHS.items()}
    return {"path": names.get(info.path, "none"), "n": info.n, "rows_redone": info.rows_redone,
            "wait_errors": info.wait_errors}


def knn_search_noalloc(rows, nbr_ids, queries, k_out: int, speedup: float, expansion: float,
                       seed: int, query_id0: int, out_ids, out_sims=None, stream=None) -> None:
    """Query search over caller-held device buffers; allocates no device memory."""
    _check_dtype(rows, "float32", "rows")
    _check_dtype(nbr_ids, "int32", "nbr_ids")
    _check_dtype(queries, "float32", "queries")
    _check_dtype(out_ids, "int64", "out_ids")
    _check_dtype(out_sims, "float32", "out_sims")
    _check(lib.knn_search_noalloc(_ptr(rows), rows.shape[0], rows.shape[1], _ptr(nbr_ids),
                                  nbr_ids.shape[1], _ptr(queries), queries.shape[0], k_out,
                                  float(speedup), float(expansion), seed, query_id0, _ptr(out_ids),
                                  _ptr(out_sims), _stream(stream)), "knn_search_noalloc")


def knn_version() -> str:
    return lib.knn_version().decode()


# --------------------------------------------------------------------------
# a small owning wrapper
# --------------------------------------------------------------------------

@dataclass
class GraphConfig:
    dim: int
    k: int = 10
    depth: int = 2
    storage: int = KNN_STORAGE_FP32
    speedup: float = 4.0
    expansion: float = 5.0
    rescore_mult: int = 4
    max_batch: int = 1024
    seed: int = 4
    capacity: int = 0

    def params(self) -> KnnParams:
        return KnnParams(self.dim, self.k, self.depth, self.storage, float(self.speedup),
                         float(self.expansion), self.rescore_mult, self.max_batch, self.seed,
                         self.capacity)


class Graph:
    """Owns one knn_graph handle; methods mirror the C calls."""

    def __init__(self, cfg: GraphConfig, init_vecs, stream=None, nbr_ids=None):
        """Exact initial graph of init_vecs, or, with nbr_ids, a restored one."""
        self.cfg = cfg
        if nbr_ids is None:
            self.handle = knn_graph_create(cfg.params(), init_vecs, stream)
        else:
            self.handle = knn_graph_restore(cfg.params(), init_vecs, nbr_ids, stream)

    def insert(self, vecs, out_ids=None, out_nbrs=None, stream=None):
        knn_graph_insert_batch(self.handle, vecs, out_ids, out_nbrs, stream)

    def query(self, vecs, k_out, query_id0, out_ids, out_sims=None, stream=None):
        knn_graph_query_batch(self.handle, vecs, k_out, query_id0, out_ids, out_sims, stream)

    def query_partitioned_ids(self, vecs, k_out, query_ids, part_offsets, out_ids, out_sims=None, stream=None):
        knn_graph_query_partitioned_ids(self.handle, vecs, k_out, query_ids, part_offsets, out_ids, out_sims,
                                        stream)

    def query_ids(self, vecs, k_out, query_ids, out_ids, out_sims=None, stream=None):
        knn_graph_query_ids(self.handle, vecs, k_out, query_ids, out_ids, out_sims, stream)

    def query_partitioned(self, vecs, k_out, query_id0, part_offsets, out_ids, out_sims=None,
                          stream=None):
        knn_graph_query_partitioned(self.handle, vecs, k_out, query_id0, part_offsets, out_ids,
                                    out_sims, stream)

    def remove(self, ids, stream=None):
        knn_graph_remove(self.handle, ids, stream)

    def set_partitions(self, labels, medoids, recompute_interval: float = 0.0, stream=None):
        knn_graph_set_partitions(self.handle, labels, medoids, recompute_interval, stream)

    def insert_distributed(self, vecs, out_ids=None, out_nbrs=None, stream=None):
        knn_graph_insert_distributed(self.handle, vecs, out_ids, out_nbrs, stream)

    def partitions(self, labels=None, medoids=None, stream=None) -> int:
        return knn_graph_get_partitions(self.handle, labels, medoids, stream)

    def reserve(self, capacity: int, headroom_bytes: int = 0, stream=None):
        knn_graph_reserve(self.handle, capacity, headroom_bytes, stream)
        self.cfg.capacity = max(self.cfg.capacity, capacity)

    def edges(self, out_ids, out_sims=None, stream=None) -> int:
        return knn_graph_get_edges(self.handle, out_ids, out_sims, stream)

    def counters(self, out, stream=None):
        knn_graph_last_counters(self.handle, out, stream)

    def stats(self) -> dict:
        return knn_graph_stats(self.handle)

    def set_timing(self, enable: bool = True):
        knn_graph_set_timing(self.handle, enable)

    def set_search(self, speedup: float, expansion: float, climb: str = "eager"):
        knn_graph_set_search(self.handle, speedup, expansion, climb)

    def last_timing(self) -> dict:
        return knn_graph_last_timing(self.handle)

    def close(self):
        if self.handle:
            knn_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over a Graph (knn_server_*).  The graph is
    owned by the server's worker until close(); submit() and wait() may be
    called from any thread (the C calls release the GIL)."""

    def __init__(self, graph: "Graph", k_out: int, max_step_points: int = 0,
                 grow_headroom_bytes: int = 0, part_offsets=None):
        """grow_headroom_bytes > 0: inserts beyond the graph's capacity grow
        it while that many bytes of device memory stay free.  part_offsets
        (host int64 [parts + 1], 0 .. the graph's n): queries run the
        partitioned search over those node ranges."""
        self.graph = graph
        self.k_out = k_out
        self.dim = graph.cfg.dim
        h = ctypes.c_void_p()
        offs = None if part_offsets is None else np.ascontiguousarray(part_offsets, dtype=np.int64)
        params = KnnServerParams(k_out, max_step_points, grow_headroom_bytes,
                                 0 if offs is None else offs.shape[0] - 1, 0,
                                 None if offs is None else offs.ctypes.data)
        _check(lib.knn_server_create(graph.handle, ctypes.byref(params), ctypes.byref(h)),
               "knn_server_create")
        self.handle = h

    def submit(self, kind: int, vecs: np.ndarray) -> int:
        """Enqueue a request of host float32 points [m, dim]; returns its id."""
        v = np.ascontiguousarray(vecs, dtype=np.float32)
        rid = ctypes.c_uint64()
        _check(lib.knn_server_submit(self.handle, kind, v.ctypes.data, v.shape[0], ctypes.byref(rid)),
               "knn_server_submit")
        return rid.value

    def wait(self, request_id: int, m: int, kind: int):
        """Block until done: (ids, sims or None, info dict).  A query's ids and
        sims are [m, k_out]; an insert's ids are its new node ids [m]."""
        ids = np.empty((m, self.k_out) if kind == KNN_REQ_QUERY else m, np.int64)
        sims = np.empty((m, self.k_out), np.float32) if kind == KNN_REQ_QUERY else None
        info = KnnRequestInfo()
        _check(lib.knn_server_wait(self.handle, request_id, ids.ctypes.data,
                                   None if sims is None else sims.ctypes.data, ctypes.byref(info)),
               "knn_server_wait")
        return ids, sims, info.as_dict()

    def stats(self) -> dict:
        out = KnnServerStats()
        _check(lib.knn_server_get_stats(self.handle, ctypes.byref(out)), "knn_server_get_stats")
        return out.as_dict()

    def close(self):
        if self.handle:
            lib.knn_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class MultiGraph:
    """Several graphs in one device arena, stepped with mixed batches
    (knn_multi_*).  Host numpy arrays in, host numpy arrays out."""

    def __init__(self, cfg: GraphConfig, n_init, capacity, init_vecs, use_graph: bool = True,
                 stream=None):
        self.cfg = cfg
        n_init = np.ascontiguousarray(n_init, dtype=np.int64)
        capacity = np.ascontiguousarray(capacity, dtype=np.int64)
        _check_dtype(init_vecs, "float32", "init_vecs")
        h = ctypes.c_void_p()
        _check(lib.knn_multi_create(ctypes.byref(cfg.params()), n_init.shape[0], n_init.ctypes.data,
                                    capacity.ctypes.data, _ptr(init_vecs), int(bool(use_graph)),
                                    _stream(stream), ctypes.byref(h)), "knn_multi_create")
        self.handle = h
        self.graphs = n_init.shape[0]

    def step(self, vecs, graph, kind, query_ids=None, with_sims: bool = False):
        v = np.ascontiguousarray(vecs, dtype=np.float32)
        gr = np.ascontiguousarray(graph, dtype=np.int32)
        kd = np.ascontiguousarray(kind, dtype=np.int32)
        m = v.shape[0]
        qid = np.ascontiguousarray(np.zeros(m, np.uint64) if query_ids is None else query_ids, dtype=np.uint64)
        out = np.empty((m, self.cfg.k), np.int64)
        sims = np.empty((m, self.cfg.k), np.float32) if with_sims else None
        _check(lib.knn_multi_step(self.handle, v.ctypes.data, gr.ctypes.data, kd.ctypes.data, qid.ctypes.data, m,
                                  out.ctypes.data, None if sims is None else sims.ctypes.data, None),
               "knn_multi_step")
        return out, sims

    def set_launch(self, search_warps: int):
        _check(lib.knn_multi_set_launch(self.handle, search_warps), "knn_multi_set_launch")

    def set_order(self, largest_first: bool):
        _check(lib.knn_multi_set_order(self.handle, int(bool(largest_first))), "knn_multi_set_order")

    def autotune(self, sample, step_caps=(512, 1024, 2048, 4096), warps=(608, 1216, 2432, 0),
                 orders=(False, True), repeats: int = 2) -> dict:
        """Pick the search launch width, the order the search takes a step's
        items in (as packed, or the largest graphs first) and the step size
        cap by timing query-only steps of `sample` (vecs, graph, query_ids:
        read-only, so the graphs do not change).  Returns the chosen settings
        and the times measured; the chosen width and order are set, the step
        cap is returned for the caller's batching (step_many)."""
        import time
        vecs, graph, qids = sample
        kind = np.ones(len(graph), np.int32)
        best, table = None, []
        for w in warps:
            self.set_launch(w)
            for lf in orders:
                self.set_order(lf)
                for cap in step_caps:
                    if cap > self.cfg.max_batch:
                        continue
                    self.step_many(vecs[:cap], graph[:cap], kind[:cap], qids[:cap], cap)  # warm (and capture)
                    t0 = time.perf_counter()
                    for _ in range(repeats):
                        self.step_many(vecs, graph, kind, qids, cap)
                    dt = (time.perf_counter() - t0) / repeats
                    rate = len(graph) / dt
                    table.append({"search_warps": w, "largest_first": bool(lf), "step_cap": cap,
                                  "items_per_s": rate})
                    if best is None or rate > best["items_per_s"]:
                        best = table[-1]
        self.set_launch(best["search_warps"])
        self.set_order(best["largest_first"])
        return {"best": best, "tried": table}

    def step_many(self, vecs, graph, kind, query_ids, cap: int):
        """Items in steps of at most `cap`, in order; the concatenated outputs."""
        outs = []
        for i in range(0, len(graph), cap):
            o, _ = self.step(vecs[i:i + cap], graph[i:i + cap], kind[i:i + cap],
                             None if query_ids is None else query_ids[i:i + cap])
            outs.append(o)
        return np.concatenate(outs)

    def size(self, graph: int):
        n, c = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.knn_multi_graph_size(self.handle, graph, ctypes.byref(n), ctypes.byref(c)),
               "knn_multi_graph_size")
        return n.value, c.value

    def edges(self, graph: int) -> np.ndarray:
        n, _ = self.size(graph)
        out = np.empty((n, self.cfg.k), np.int64)
        _check(lib.knn_multi_get_edges(self.handle, graph, out.ctypes.data, None), "knn_multi_get_edges")
        return out

    def close(self):
        if self.handle:
            lib.knn_multi_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
