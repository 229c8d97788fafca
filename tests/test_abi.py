"""The C-ABI library loads and exports every entry point include/cello.h
declares (no GPU needed: nothing is called)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "cello.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cello_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("cello_octree_build", "cello_refine_flags", "cello_ghost_refresh", "cello_hydro_step"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1810_01319_gb300 import build
    build.build()
    from paper_1810_01319_gb300 import _lib
    L = _lib.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) == set(_lib.SIGNATURES)


def test_product_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1810_01319_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(_lib.CelloError):
        _lib.lib()
