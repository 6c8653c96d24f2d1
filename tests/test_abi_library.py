"""The C-ABI library builds, loads and exports every entry point that
include/ara.h declares (no GPU needed: nothing here launches device work)."""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ara.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ARA_API\s+[\w\s\*]*?\b(ara_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ara_load_yet", "ara_load_elts", "ara_run_layer", "ara_pml_tvar"):
        assert required in names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1501_06326_gb300 import build

    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        if not os.path.exists(build.LIB):
            pytest.skip("nvcc not available and libara.so not built")
        return build.LIB
    return build.build()


def test_library_exports_every_declared_function(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_mirrors_the_header(lib_path):
    from paper_1501_06326_gb300 import ara

    assert sorted(ara.EXPORTED) == declared_functions()
    lib = ara.load_library(lib_path)
    for name in ara.EXPORTED:
        assert getattr(lib, name).argtypes is not None or name == "ara_last_error"


def test_binding_rejects_wrong_dtypes():
    import numpy as np

    from paper_1501_06326_gb300 import ara

    with pytest.raises(TypeError):
        ara._ptr(np.zeros(4, np.int32), np.int64)
    with pytest.raises(ValueError):
        ara._ptr(np.zeros((4, 4), np.int64)[:, 0], np.int64)
