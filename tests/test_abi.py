"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/alelb.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_2002_04353_gb300 import alelb, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "alelb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(alelb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["alelb_mesh_create", "alelb_mesh_move", "alelb_lb_init", "alelb_lb_step",
              "alelb_moments", "alelb_forces"]:
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert sorted(_declared()) == sorted(alelb.EXPORTS)


def test_binding_fails_loudly_without_the_library(tmp_path):
    import pytest
    old = alelb._lib
    alelb._lib = None
    try:
        with pytest.raises(RuntimeError):
            alelb.load(str(tmp_path / "missing.so"))
    finally:
        alelb._lib = old
