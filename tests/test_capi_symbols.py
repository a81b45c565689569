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


def test_build_targets_sm103a_in_tree(monkeypatch):
    """Every translation unit compiles for sm_103a alone (one -gencode), with line info, into
    the package's own _lib directory; the C++ unit is compiled as CUDA."""
    from paper_2112_04167_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.dirname(build.LIB) == os.path.join(ROOT, "paper_2112_04167_gb300", "_lib")
    seen = []

    class R:
        returncode, stdout, stderr = 0, "", ""

    monkeypatch.setattr(build.subprocess, "run", lambda cmd, **kw: (seen.append(cmd), R())[1])
    for src in ("k_sipg.cu", "basis.cpp"):
        build._compile(src, "nvcc", [])
    for cmd in seen:
        assert cmd.count("-gencode") == 1 and "arch=compute_103a,code=sm_103a" in cmd
        assert "-lineinfo" in cmd and "-O3" in cmd
    assert seen[1][-2:] == ["-x", "cu"]
    assert all(s in build.SOURCES for s in ("imex.cu", "k_sipg_line32.cu", "k_sipg_line64.cu", "basis.cpp"))
