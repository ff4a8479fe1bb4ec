"""The C ABI library builds, loads, exports every entry point that
include/knn_graph.h declares, and rejects bad arguments before any device
work.  No GPU: nothing here launches a kernel."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "knn_graph.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"KNN_API\s+[\w\s\*]+?\b(knn_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def knn():
    from paper_1602_06819_gb300 import build
    build.build()
    from paper_1602_06819_gb300 import knn as module
    return module


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("knn_graph_create", "knn_graph_insert_batch", "knn_graph_query_batch",
                     "knn_graph_remove", "knn_graph_get_edges", "knn_exact_graph",
                     "knn_graph_destroy", "knn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(knn):
    declared = declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", knn._LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    assert set(declared) == set(knn.EXPORTED)
    # nothing but the ABI is exported from our own code
    ours = {s for s in exported if s.startswith("knn_")}
    assert ours == set(declared)


def test_struct_layouts_match_header(knn):
    assert ctypes.sizeof(knn.KnnParams) == 56
    assert ctypes.sizeof(knn.KnnStats) == 15 * 8


def _params(knn, **kw):
    base = dict(dim=16, k=10, depth=2, storage=0, speedup=4.0, expansion=5.0, rescore_mult=4,
                max_batch=8, seed=1, capacity=100)
    base.update(kw)
    return knn.KnnParams(*(base[f] for f, _ in knn.KnnParams._fields_))


@pytest.mark.parametrize("bad,status", [
    (dict(dim=0), -7), (dict(dim=257), -7), (dict(k=0), -7), (dict(k=33), -7),
    (dict(depth=0), -7), (dict(depth=6), -7), (dict(storage=5), -1), (dict(speedup=0.0), -1),
    (dict(speedup=float("inf")), -1), (dict(expansion=float("nan")), -1),
    (dict(storage=1, rescore_mult=0), -7), (dict(storage=2, k=32, rescore_mult=5), -7),
    (dict(max_batch=0), -1), (dict(capacity=10), -3)])
def test_create_rejects_bad_parameters(knn, bad, status):
    X = np.zeros((20, 16), np.float32)
    h = ctypes.c_void_p()
    st = knn.lib.knn_graph_create(ctypes.byref(_params(knn, **bad)), X.ctypes.data, 20, None,
                                  ctypes.byref(h))
    assert st == status
    assert h.value is None
    assert knn.lib.knn_last_error().decode()


def test_create_needs_k_plus_one_points(knn):
    X = np.zeros((10, 16), np.float32)
    h = ctypes.c_void_p()
    st = knn.lib.knn_graph_create(ctypes.byref(_params(knn)), X.ctypes.data, 10, None, ctypes.byref(h))
    assert st == knn.KNN_ERR_INVALID_ARG and "k + 1" in knn.lib.knn_last_error().decode()


def test_null_handles_are_rejected(knn):
    X = np.zeros((4, 16), np.float32)
    ids = np.zeros(4, np.int64)
    assert knn.lib.knn_graph_insert_batch(None, X.ctypes.data, 4, None, None, None) == -1
    assert knn.lib.knn_graph_query_batch(None, X.ctypes.data, 4, 1, 0, ids.ctypes.data, None, None) == -1
    assert knn.lib.knn_graph_remove(None, ids.ctypes.data, 4, None) == -1
    n_out = ctypes.c_int64()
    assert knn.lib.knn_graph_get_edges(None, ids.ctypes.data, None, 4, ctypes.byref(n_out), None) == -1
    knn.lib.knn_graph_destroy(None)  # no-op


def test_every_handle_entry_point_rejects_a_null_handle(knn):
    """Each call that takes a graph, server or multi-graph handle refuses a
    null one with KNN_ERR_INVALID_ARG before touching any other argument
    (the other pointers here are valid host buffers, never read)."""
    lib = knn.lib
    X = np.zeros((4, 16), np.float32)
    i64 = np.zeros(64, np.int64)
    i32 = np.zeros(64, np.int32)
    u64 = np.zeros(64, np.uint64)
    f32 = np.zeros(64, np.float32)
    x, a, b, u, f = X.ctypes.data, i64.ctypes.data, i32.ctypes.data, u64.ctypes.data, f32.ctypes.data

    class Lib:  # addresses cast to whatever pointer type a function's argtypes name
        def __getattr__(self, name):
            fn = getattr(knn.lib, name)

            def call(*args):
                types = fn.argtypes or [None] * len(args)
                conv = [ctypes.cast(ctypes.c_void_p(v), t)
                        if isinstance(v, int) and t is not None and issubclass(t, ctypes._Pointer) else v
                        for v, t in zip(args, types)]
                return fn(*conv)
            return call
    lib = Lib()
    calls = {
        "knn_graph_query_ids": lambda: lib.knn_graph_query_ids(None, x, 4, 1, u, a, f, None),
        "knn_graph_query_partitioned": lambda: lib.knn_graph_query_partitioned(
            None, x, 4, 1, 0, a, 2, a, f, None),
        "knn_graph_query_partitioned_ids": lambda: lib.knn_graph_query_partitioned_ids(
            None, x, 4, 1, u, a, 2, a, f, None),
        "knn_graph_set_partitions": lambda: lib.knn_graph_set_partitions(None, b, a, 2, 0.1, None),
        "knn_graph_insert_distributed": lambda: lib.knn_graph_insert_distributed(None, x, 4, a, None, None),
        "knn_graph_get_partitions": lambda: lib.knn_graph_get_partitions(None, b, a, a, None),
        "knn_graph_last_counters": lambda: lib.knn_graph_last_counters(None, a, 4, None),
        "knn_graph_set_timing": lambda: lib.knn_graph_set_timing(None, 1),
        "knn_graph_last_timing": lambda: lib.knn_graph_last_timing(None, f, 4),
        "knn_graph_stats": lambda: lib.knn_graph_stats(None, a),
        "knn_graph_reserve": lambda: lib.knn_graph_reserve(None, 1000, 0, None),
        "knn_server_submit": lambda: lib.knn_server_submit(None, 0, x, 1, u),
        "knn_server_wait": lambda: lib.knn_server_wait(None, 1, a, f, None),
        "knn_server_get_stats": lambda: lib.knn_server_get_stats(None, a),
        "knn_multi_step": lambda: lib.knn_multi_step(None, x, b, b, u, 4, a, f, None),
        "knn_multi_set_launch": lambda: lib.knn_multi_set_launch(None, 4),
        "knn_multi_set_order": lambda: lib.knn_multi_set_order(None, 1),
        "knn_multi_graph_size": lambda: lib.knn_multi_graph_size(None, 0, a, a),
        "knn_multi_get_edges": lambda: lib.knn_multi_get_edges(None, 0, a, None),
    }
    assert set(calls) <= set(declared_functions())
    for name, call in calls.items():
        assert call() == knn.KNN_ERR_INVALID_ARG, name
        assert knn.lib.knn_last_error().decode(), name
    sh = ctypes.c_void_p()
    assert knn.lib.knn_server_create(None, None, ctypes.byref(sh)) == knn.KNN_ERR_INVALID_ARG
    assert sh.value is None
    knn.lib.knn_server_destroy(None)  # no-op
    knn.lib.knn_multi_destroy(None)   # no-op


def test_exact_graph_rejects_bad_sizes(knn):
    X = np.zeros((5, 8), np.float32)
    ids = np.zeros((5, 4), np.int64)
    assert knn.lib.knn_exact_graph(X.ctypes.data, 5, 8, 0, ids.ctypes.data, None, None) == -7
    assert knn.lib.knn_exact_graph(X.ctypes.data, 5, 8, 5, ids.ctypes.data, None, None) == -1
    assert knn.lib.knn_exact_graph(X.ctypes.data, 5, 300, 2, ids.ctypes.data, None, None) == -7


def test_exact_path_setting_checks_its_arguments(knn):
    assert knn.lib.knn_exact_set_path(3) == -1
    assert knn.lib.knn_exact_set_path(-1) == -1
    assert knn.lib.knn_exact_last_info(None) == -1
    for name in ("cuda_cores", "tensor_cores", "auto"):
        knn.knn_exact_set_path(name)
    assert ctypes.sizeof(knn.KnnExactInfo) == 24
    info = knn.knn_exact_last_info()   # no build ran on this thread yet
    assert info["n"] == 0 and info["rows_redone"] == 0


def test_set_search_checks_its_arguments(knn):
    assert knn.lib.knn_graph_set_search(None, 4.0, 5.0, 0) == -1


def test_binding_raises_with_message(knn):
    with pytest.raises(knn.KnnError) as e:
        knn.knn_graph_create(_params(knn, k=0), np.zeros((20, 16), np.float32), stream=0)
    assert e.value.status == knn.KNN_ERR_UNSUPPORTED


def test_binding_checks_dtypes_and_layout_before_the_call(knn):
    """Argument marshalling refuses what the C ABI cannot take (the ABI sees
    only pointers): a wrong element type or a strided view, before any call."""
    p = _params(knn)
    with pytest.raises(TypeError):
        knn.knn_graph_create(p, np.zeros((20, 16), np.float64), stream=0)
    with pytest.raises(ValueError):
        knn.knn_graph_create(p, np.zeros((20, 32), np.float32)[:, ::2], stream=0)
    with pytest.raises(TypeError):
        knn.knn_graph_restore(p, np.zeros((20, 16), np.float32), np.zeros((20, 10), np.int32), stream=0)
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        knn.knn_graph_create(p, torch.zeros(16, 20).t(), stream=0)
    with pytest.raises(TypeError):
        knn.knn_graph_create(p, torch.zeros(20, 16, dtype=torch.float16), stream=0)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """The binding has no fallback: without the library, import fails."""
    import importlib
    import paper_1602_06819_gb300.build as b
    monkeypatch.setattr(b, "LIB", str(tmp_path / "absent.so"))
    import paper_1602_06819_gb300.knn as k
    monkeypatch.setattr(k, "_LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        k._load_library()
    importlib.reload(b)


def test_noalloc_search_checks_alignment_before_any_device_work(knn):
    """Rows and queries are read with 16-byte loads: a misaligned pointer is
    refused by pointer arithmetic alone, before any CUDA call (here there is
    no GPU, and the pointers are never dereferenced)."""
    lib = knn.lib
    base = 1 << 20
    args = dict(rows=base, n=1000, dim=16, nbr=base, k=4, q=base, m=8, k_out=4, ids=base,
                sims=base)

    def call(**kw):
        a = dict(args, **kw)
        return lib.knn_search_noalloc(a["rows"], a["n"], a["dim"], a["nbr"], a["k"], a["q"], a["m"],
                                      a["k_out"], 4.0, 5.0, 1, 0, a["ids"], a["sims"], None)

    for bad in (dict(rows=base + 4), dict(q=base + 8), dict(nbr=base + 2), dict(ids=base + 4),
                dict(sims=base + 1)):
        assert call(**bad) == knn.KNN_ERR_INVALID_ARG, bad
        msg = lib.knn_last_error().decode()
        assert "boundary" in msg or "aligned" in msg, msg
