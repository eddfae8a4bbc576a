"""The C-ABI library loads and exports every symbol include/*.h declares (CPU only, no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2105_13611_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_five_entry_points():
    names = declared_functions()
    for n in ["load_linelist", "set_atmosphere_grid", "synth_opacity", "build_odf", "synth_spectrum"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert declared_functions() <= exported


def test_binding_names_match_header(lib_path):
    from paper_2105_13611_gb300 import binding
    assert set(binding.EXPORTED) <= declared_functions()
    lib = binding.load_library(lib_path)
    assert lib.mpsa_version().startswith(b"mpsa")
    g = binding.LGrid(300.0, 400.0, 2e6)
    assert lib.mpsa_grid_size(ctypes.byref(g)) == 575365
