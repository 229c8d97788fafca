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


def test_mesh_desc_layout_matches_the_header(tmp_path):
    """The binding's ctypes view of cello_mesh_desc has the size and field
    offsets the C compiler gives the header's struct."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1810_01319_gb300 import _lib
    fields = [f for f, _ in _lib.MeshDesc._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("{f} %zu\\n", offsetof(cello_mesh_desc, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "cello.h"\nint main(void) {\n'
                   '  printf("sizeof %zu\\n", sizeof(cello_mesh_desc));\n' + body + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(out["sizeof"]) == ctypes.sizeof(_lib.MeshDesc)
    for f in fields:
        assert int(out[f]) == getattr(_lib.MeshDesc, f).offset, f
