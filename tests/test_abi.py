"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(aimx_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2009_02281_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    decl = _declared()
    assert "aimx_setup" in decl and "aimx_matvec" in decl
    for name in sorted(decl):
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2009_02281_gb300 import aimx
    bound = {n for n, _, _ in aimx._SIGS}
    assert _declared() <= bound


def test_status_strings_without_gpu():
    from paper_2009_02281_gb300 import aimx
    lib = aimx.load(build_if_missing=True)
    assert lib.aimx_status_string(0) == b"ok"
    assert lib.aimx_status_string(-3) == b"stencil outside the grid"


def test_setup_rejects_bad_arguments_without_gpu():
    from paper_2009_02281_gb300 import aimx
    lib = aimx.load(build_if_missing=True)
    out = ctypes.c_void_p()
    assert lib.aimx_setup(None, None, None, 2, ctypes.byref(out)) == -1
