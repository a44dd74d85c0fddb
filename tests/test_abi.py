"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/pz.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pz.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pz_[a-z0-9_]+)\s*\(", src)))


def test_header_compiles_as_c_and_cpp(tmp_path):
    for lang, cc in (("c", "gcc"), ("c++", "g++")):
        r = subprocess.run([cc, "-x", lang, "-fsyntax-only", "-Wall", "-Werror", HEADER], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol():
    from paper_2607_24141_gb300 import build
    try:
        path = build.build()
    except (RuntimeError, FileNotFoundError) as e:  # pragma: no cover
        pytest.fail("libpz.so failed to build: %s" % e)
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    import paper_2607_24141_gb300 as pz
    assert sorted(pz.EXPORTED) == names


def test_binding_has_no_cpu_fallback():
    import paper_2607_24141_gb300 as pz
    src = open(pz.__file__).read()
    assert "oracle" not in src
