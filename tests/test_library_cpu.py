"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, and
exports every symbol that include/nqs.h declares. No GPU call is made."""
import ctypes
import os
import re

import pytest

from paper_2507_19276_gb300 import build, nqs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "nqs.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(nqs_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_binding_names():
    assert declared_symbols() == sorted(nqs.exported_symbols())


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
