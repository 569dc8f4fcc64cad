"""The C ABI library loads without a GPU and exports every entry point include/leb.h declares."""
import ctypes as C
import os
import re

import pytest

from paper_2607_01203_b300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "leb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(leb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_expected_calls():
    names = declared_symbols()
    for required in ("leb_create", "leb_destroy", "leb_bounds", "leb_bounds_backward", "leb_workspace_size",
                     "leb_autotune", "leb_graph_capture", "leb_proposer_train_step", "leb_zonotope_map"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = binding.lib()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTS) <= set(declared_symbols())


def test_host_side_validation_without_gpu():
    lib = binding.lib()
    assert lib.leb_version().startswith(b"leb-b300")
    assert lib.leb_status_string(-3) == b"workspace missing or too small"
    h = C.c_void_p()
    assert lib.leb_create(None, C.byref(h)) == binding.LEB_OK - 1          # NULL spec
    assert lib.leb_destroy(None) == -1
    assert lib.leb_zonotope_map(None, None, -1, 0.0, None, None, None) == -1
    assert lib.leb_zonotope_map(None, None, 0, -1.0, None, None, None) == -1
    assert lib.leb_zonotope_map(None, None, 0, 0.0, None, None, None) == 0  # nothing to do
    assert lib.leb_graph_launch(None, None) == -1
