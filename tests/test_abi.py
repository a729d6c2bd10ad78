"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/mnemonic.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "mnemonic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mn_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2206_09983_b300 import build
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None and not os.path.exists(build.LIB):
        pytest.fail("nvcc missing and libmnemonic.so not built")
    return build.build()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("mn_create_graph", "mn_register_query", "mn_insert_batch", "mn_delete_batch",
              "mn_fetch_embeddings", "mn_count_static", "mn_destroy_graph", "mn_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export(lib_path):
    from paper_2206_09983_b300 import mnemonic
    assert set(mnemonic.EXPORTS) == set(declared_entry_points())
    mnemonic.load()   # resolves every signature without a device


def test_create_error_without_device_is_reported(lib_path):
    """mn_create_graph rejects bad configs on the host, before touching CUDA."""
    from paper_2206_09983_b300 import mnemonic as M
    lib = M.load()
    cfg = M._Config(0, 1, None, 0, 16, 16, 0, 0, 1, 0, None)
    h = ctypes.c_void_p()
    st = lib.mn_create_graph(ctypes.byref(cfg), ctypes.byref(h))
    assert st == -1 and not h.value
    assert b"num_vertices" in lib.mn_last_error(None)
