"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/*.h declares; host-side argument checks need no GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(prdf_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_2404_08299_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["prdf_graph_create", "prdf_graph_apply_batch", "prdf_partition", "prdf_initial_affected",
                     "prdf_expand_affected", "prdf_pagerank_static", "prdf_pagerank_dfp"]:
        assert required in names


def test_every_declared_symbol_is_exported(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    import paper_2404_08299_gb300 as prdf
    assert set(declared_functions()) <= set(prdf._SIGNATURES)


def test_params_default_are_the_papers_constants(built_lib):
    import paper_2404_08299_gb300 as prdf
    p = prdf._Params()
    built_lib.prdf_params_default(ctypes.byref(p))
    assert (p.alpha, p.tol, p.tau_f, p.tau_p, p.max_iter) == (0.85, 1e-10, 1e-6, 1e-6, 500)
    assert p.precision == prdf.PRDF_FP64 and p.accumulate == prdf.PRDF_ACC_EXACT and p.prune == 1
    assert p.expand_pull == 1 / 16 and p.expand_list == -1 and p.stream is None


def test_graph_create_rejects_bad_sizes_without_touching_the_gpu(built_lib):
    f = built_lib.prdf_graph_create
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint,
                  ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert f(0, None, None, None, 0, 1, None, ctypes.byref(out)) == -1
    assert f(5, None, None, None, -1, 1, None, ctypes.byref(out)) == -1
    assert f(5, None, None, None, 3, 1, None, ctypes.byref(out)) == -1  # m0 > 0 with NULL arrays
    built_lib.prdf_last_error.restype = ctypes.c_char_p
    assert b"bad arguments" in built_lib.prdf_last_error()
    built_lib.prdf_strerror.restype = ctypes.c_char_p
    assert built_lib.prdf_strerror(-1) == b"invalid argument"


def test_release_cached_memory_without_a_pool_is_a_no_op(built_lib):
    # no device allocation has happened in this process, so no pool exists to trim
    built_lib.prdf_release_cached_memory.restype = ctypes.c_int
    assert built_lib.prdf_release_cached_memory() == 0


def test_product_path_has_no_cpu_fallback(monkeypatch, tmp_path):
    import paper_2404_08299_gb300 as prdf
    monkeypatch.setattr(prdf, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(prdf, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        prdf.lib()


def test_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2404_08299_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "oracle.c" not in text, path
