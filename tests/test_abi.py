"""The C ABI library loads and exports every entry point include/grass.h
declares; the binding declares the same names.  No GPU needed (no compute
call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grass.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grass_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import paper_1911_04382_gb300 as G
    return G.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("grass_build_tree", "grass_embed", "grass_filter", "grass_densify",
                 "grass_pcg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_exposes_the_same_names(libpath):
    import paper_1911_04382_gb300 as G
    missing = [n for n in _declared() if not hasattr(G, n)]
    assert not missing, missing


def test_null_arguments_are_rejected_without_a_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.grass_ctx_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.grass_ctx_create.restype = ctypes.c_int
    assert L.grass_ctx_create(None, None) == 1          # GRASS_ERR_INVALID
    L.grass_tree_info.argtypes = [ctypes.c_void_p] * 4
    L.grass_tree_info.restype = ctypes.c_int
    assert L.grass_tree_info(None, None, None, None) == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_1911_04382_gb300.binding as B
    monkeypatch.setattr(B, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        B.lib()


def test_server_footprint_is_host_only_and_monotone(libpath):
    import paper_1911_04382_gb300 as G
    f = G.grass_server_footprint
    assert f(0, 10, 8, 1) == -1 and f(10, -1, 8, 1) == -1 and f(10, 10, 0, 1) == -1
    base = f(10_000, 50_000, 8, 3)
    # at least the request's own inputs: CSR, h0, v0, b, x
    n, nnz, r, R = 10_000, 50_000, 8, 3
    assert base >= 8 * (n + 1) + 12 * nnz + 8 * n * r * R + 8 * n * R + 16 * n
    assert f(20_000, 50_000, 8, 3) > base and f(10_000, 90_000, 8, 3) > base
    assert f(10_000, 50_000, 16, 3) > base and f(10_000, 50_000, 8, 4) > base


def test_kernel_source_hash_ignores_comments():
    """The capture records in profiles/traffic.json stay valid across comment
    edits but not across code edits."""
    import bench
    src = {"a": "int x; // one\n/* block\n comment */\nint y;\n\n", "b": "float z;\n"}
    base = bench.KERNEL_SOURCES
    try:
        bench.KERNEL_SOURCES = ["a", "b"]
        h0 = bench.kernel_sources_hash(lambda s: src[s])
        src["a"] = "int x;  // two\n\nint y;\n"
        assert bench.kernel_sources_hash(lambda s: src[s]) == h0
        src["a"] = "int x; int y;\n"
        assert bench.kernel_sources_hash(lambda s: src[s]) != h0
    finally:
        bench.KERNEL_SOURCES = base
