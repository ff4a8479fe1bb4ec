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
