"""The C-ABI library loads (no GPU needed) and exports every function that
include/pm.h declares; the Python binding declares the same set."""
import ctypes
import os
import re

import paper_1904_09538_gb300 as pm
from paper_1904_09538_gb300 import _lib

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pm.h")


def declared():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_0-9]+)\s*\(", text)))


def test_header_symbols_exported():
    names = declared()
    assert len(names) >= 25, names
    so = ctypes.CDLL(_lib.SO)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert sorted(_lib.SIGNATURES) == declared()


def test_registry_round_trip():
    names = pm.kernel_names()
    assert len(names) == len(set(names)) >= 26
    text = open(HDR).read()
    for n in names:      # every registered kernel is documented in the header
        assert '"%s"' % n in text, n
    for i, n in enumerate(names):
        assert pm.kernel_lookup(n) == i
