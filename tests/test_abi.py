"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/hb.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(hb_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["hb_init", "hb_query", "hb_build_blocks", "hb_diag", "hb_classify", "hb_destroy", "hb_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1709_03005_gb300 import build_ext, hb
    path = build_ext.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(hb.EXPORTS) <= set(_declared())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1709_03005_gb300 import hb
    import pytest
    saved = hb._lib
    hb._lib = None
    try:
        with pytest.raises(RuntimeError):
            hb.load(str(tmp_path / "missing.so"))
    finally:
        hb._lib = saved
