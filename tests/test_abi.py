"""The C-ABI library builds, loads and exports every entry point include/*.h
declares (no GPU: nothing is called that would need one)."""
import ctypes
import glob
import os
import re

import pytest

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(morph_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2305_03018_gb300 import build_lib
    path = build_lib.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 12, declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2305_03018_gb300 import morph
    declared = _declared()
    assert declared <= set(morph._SIGS), declared - set(morph._SIGS)
    for n in declared:
        assert hasattr(morph, n), n


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2305_03018_gb300 import morph
    saved = morph._lib
    morph._lib = None
    try:
        with pytest.raises(RuntimeError):
            morph.load_library(str(tmp_path / "missing.so"))
    finally:
        morph._lib = saved
