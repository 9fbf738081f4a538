"""The C-ABI library builds, loads without a GPU and exports every function include/relo.h
declares; the ctypes binding names exactly those functions.  No compute call is made."""
import ctypes
import os
import re

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            s = open(os.path.join(inc, f)).read()
            s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
            s = re.sub(r"//[^\n]*", "", s)
            names |= set(re.findall(r"\b(relo_[a-z0-9_]+)\s*\(", s))
    return names


def test_header_declares_the_binding_names():
    declared = _declared()
    assert len(declared) > 40
    assert declared == set(B.EXPORTED)


def test_library_loads_and_exports_every_declared_function():
    build.build()
    L = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert B.lib() is not None
