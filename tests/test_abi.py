"""The C ABI without a GPU: libfewha.so builds for sm_103a, loads, and exports
every function that include/fewha.h declares; the Python binding names the
same set.  No compute call is made."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fewha.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|long|double|void|char)\s*\**\s*(fewha_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2011_06842_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("fewha_create", "fewha_apply_op", "fewha_solve", "fewha_rhs", "fewha_destroy",
                 "fewha_apply_op_multi", "fewha_conv3x3_fwd", "fewha_deflate_warm_start"):
        assert must in names
    assert len(names) >= 29


def test_library_exports_every_declared_function(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_the_same_set(libpath):
    from paper_2011_06842_gb300 import fewha
    fewha.load_library(libpath)
    assert sorted(fewha.exported_symbols()) == declared_functions()


def test_strerror_without_a_device(libpath):
    from paper_2011_06842_gb300 import fewha
    lib = fewha.load_library(libpath)
    assert lib.fewha_strerror(0) is not None
    assert lib.fewha_strerror(-8) != lib.fewha_strerror(0)
