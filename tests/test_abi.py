"""CPU checks of the C-ABI boundary: the library builds, loads and exports every symbol that
include/bv.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(bv_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["bv_create", "bv_destroy", "bv_set_data", "bv_build_blocks", "bv_select_neighbors",
              "bv_loglik", "bv_mle", "bv_simulate", "bv_strerror"]:
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2410_04477_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert lib.bv_strerror  # resolvable
    lib.bv_strerror.restype = ctypes.c_char_p
    assert lib.bv_strerror(4).decode().startswith("covariance")


def test_binding_names_match_header():
    from paper_2410_04477_gb300 import _build
    _build.build()
    from paper_2410_04477_gb300 import bv
    assert set(bv.EXPORTED) == set(_declared())


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "bv_copy", os.path.join(ROOT, "paper_2410_04477_gb300", "bv.py"))
    mod = importlib.util.module_from_spec(spec)
    # load a copy of the binding from a directory with no built library next to it
    src = open(os.path.join(ROOT, "paper_2410_04477_gb300", "bv.py")).read()
    p = tmp_path / "bv.py"
    p.write_text(src)
    spec = importlib.util.spec_from_file_location("bv_copy", str(p))
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
