"""The C-ABI library builds, loads and exports every declared symbol (no
GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:int|void|const\s+char\s*\*)\s*\**\s*(sg_\w+)\s*\(",
                            src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1605_01421_gb300 import binding
    try:
        return binding.build()
    except FileNotFoundError:
        pytest.skip("nvcc not available")


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("sg_model_create", "sg_set_events", "sg_run", "sg_run_host",
              "sg_model_destroy", "sg_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name), name


def test_strerror_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.sg_strerror.restype = ctypes.c_char_p
    assert L.sg_strerror(0) == b"ok"
    assert b"more individuals" in L.sg_strerror(-2)


def test_binding_lists_the_exports():
    from paper_1605_01421_gb300 import binding
    assert set(binding.EXPORTS) <= set(_declared())


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1605_01421_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "siminf_oracle" not in text, fn
