"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point the headers in include/ declare (no compute calls here)."""

import ctypes
import os
import re
import subprocess

import pytest

from paper_2209_00103_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header=None):
    inc = os.path.join(ROOT, "include")
    names = [header] if header else sorted(f for f in os.listdir(inc) if f.endswith(".h"))
    text = "".join(open(os.path.join(inc, f)).read() for f in names)
    return sorted(set(re.findall(r"^int\s+(gga_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols("gga.h")
    for name in ["gga_create", "gga_insert", "gga_read", "gga_write", "gga_flatten", "gga_size", "gga_destroy"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(gga_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_names_match_header():
    from paper_2209_00103_gb300 import gga
    assert sorted(gga.EXPORTED) == declared_symbols()



@pytest.mark.parametrize("header", sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")))
def test_headers_compile_alone_as_c_and_cpp(header, tmp_path):
    # The C ABI's headers are usable from plain C (C99) and from C++ with
    # nothing else included first.
    src = tmp_path / "t.c"
    src.write_text(f'#include "{header}"\nint main(void) {{ return 0; }}\n')
    inc = "-I" + os.path.join(ROOT, "include")
    for cmd in (["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", inc, "-fsyntax-only", str(src)],
                ["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", inc, "-x", "c++", "-fsyntax-only", str(src)]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
