"""The C-ABI library loads and exports every function the public headers
declare (no compute calls: CPU only)."""
from __future__ import annotations

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in ("bilu.h", "bilu_tuning.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(libbilu):
    from paper_1703_01325_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 20
    for name in sorted(names):
        assert hasattr(libbilu, name), f"libbilu.so does not export {name}"
    assert names == set(_lib.SIGNATURES), names ^ set(_lib.SIGNATURES)


def test_library_is_sm103a_build():
    from paper_1703_01325_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
