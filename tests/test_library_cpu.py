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


def test_binding_structs_match_the_header_layout(tmp_path):
    """sizeof and field offsets of the C structs, compiled from the header,
    against the ctypes mirrors the binding passes across the boundary."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    fields = {"nqs_options": [f for f, _ in nqs.Options._fields_],
              "nqs_energy_summary": [f for f, _ in nqs.EnergySummary._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nqs.h"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                text=True).stdout.splitlines())
    for st, cls in (("nqs_options", nqs.Options), ("nqs_energy_summary", nqs.EnergySummary)):
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
