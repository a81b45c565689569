"""The C-ABI library builds here (cross-compiled for sm_103a) and exports every
symbol that include/imex.h declares; no compute call is made without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "imex.h")).read()
    pat = r"^\s*(?:imex_status|void|const char\*|long long|int)\s+(imex_\w+)\s*\("
    return sorted(set(re.findall(pat, src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_04167_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_binding(lib):
    from paper_2112_04167_gb300 import imex
    assert _declared() == imex.exported_symbols()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_refuses_missing_library(tmp_path):
    from paper_2112_04167_gb300 import imex
    with pytest.raises(ImportError):
        imex.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(imex.load, "__wrapped__") else \
            _load_fresh(imex, str(tmp_path / "nope.so"))


def _load_fresh(imex, path):
    saved = imex._lib
    imex._lib = None
    try:
        return imex.load(path)
    finally:
        imex._lib = saved
