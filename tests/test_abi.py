"""The C-ABI library loads and exports every function declared in include/cgks.h
(no compute calls: runs without a GPU)."""
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def declared():
    txt = open(os.path.join(ROOT, "include", "cgks.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cgks_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("cgks_create_mesh", "cgks_set_state", "cgks_step", "cgks_get_state"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2508_08965_gb300 as p
    L = p.lib()
    for n in declared():
        assert hasattr(L, n), n
    assert set(declared()) >= set(p.binding.EXPORTS)


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2508_08965_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*|/\*.*?\*/", "", src, flags=re.S), f


def test_header_is_plain_c():
    """include/cgks.h compiles as C11 (plain pointers and sizes, no C++ in
    the signatures) and as C++"""
    import shutil
    import subprocess
    import pytest
    hdr = os.path.join(ROOT, "include", "cgks.h")
    gcc, gxx = shutil.which("gcc"), shutil.which("g++")
    if gcc is None or gxx is None:
        pytest.skip("no host compiler")
    for cmd in ([gcc, "-fsyntax-only", "-std=c11", "-Wall", "-Werror", "-x", "c", hdr],
                [gxx, "-fsyntax-only", "-std=c++17", "-Wall", "-Werror", "-x", "c++", hdr]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
