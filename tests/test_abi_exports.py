"""The C-ABI library loads and exports every entry point include/crkdg.h
declares (no GPU needed: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(crkdg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2307_06471_gb300 import build, binding
    build.build()
    L = binding.lib()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    assert len(declared()) >= 20
    assert b"sm_103a" in L.crkdg_version()


def test_binding_covers_the_abi():
    from paper_2307_06471_gb300 import binding
    assert set(declared()) == set(binding._SIGS)
