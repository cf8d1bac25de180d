"""The C-ABI library builds, loads and exports every symbol include/rewl.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(rewl_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_builds_and_exports_header_symbols():
    from paper_1508_02748_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert "rewl_create" in declared and "rewl_get_lng" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1508_02748_gb300 import rewl
    assert sorted(rewl.SIGNATURES) == _declared()


def test_workspace_size_and_validation_without_gpu():
    import paper_1508_02748_gb300 as P
    lib = P.load_library()
    n = ctypes.c_size_t(0)
    c = P.Config(L=8, n_win_E=3, n_win_M=3, walkers_per_window=4).to_c()
    assert lib.rewl_workspace_size(ctypes.byref(c), ctypes.byref(n)) == 0
    # tables: 36 walkers x 44 x 44 bins, rounded to 64 entries, 8 + 4 bytes per bin
    assert n.value >= 36 * 1984 * 12
    bad = P.Config(L=3).to_c()
    assert lib.rewl_workspace_size(ctypes.byref(bad), ctypes.byref(n)) == -1
    assert b"L must be" in lib.rewl_last_error(None)
    bad = P.Config(L=8, flatness=1.5).to_c()
    assert lib.rewl_workspace_size(ctypes.byref(bad), ctypes.byref(n)) == -1
    # ln f must stay a power of two (every ln g exact): 0.7 and a factor 0.3 are refused
    for kw in (dict(lnf_init=0.7), dict(lnf_factor=0.3), dict(lnf_init=2.0 ** -70)):
        bad = P.Config(L=8, **kw).to_c()
        assert lib.rewl_workspace_size(ctypes.byref(bad), ctypes.byref(n)) == -1
        assert b"power" in lib.rewl_last_error(None)
    for kw in (dict(lnf_init=4.0), dict(lnf_factor=0.25), dict(lnf_init=2.0 ** -27)):
        ok = P.Config(L=8, **kw).to_c()
        assert lib.rewl_workspace_size(ctypes.byref(ok), ctypes.byref(n)) == 0
    # placement knobs: unknown values are refused; a register lattice needs N <= 64
    for kw in (dict(table_mode=3), dict(lattice_mode=-1), dict(L=12, lattice_mode=P.LATTICE_REGISTER)):
        bad = P.Config(**{"L": 8, **kw}).to_c()
        assert lib.rewl_workspace_size(ctypes.byref(bad), ctypes.byref(n)) == -1
    for kw in (dict(lattice_mode=P.LATTICE_REGISTER), dict(L=12, lattice_mode=P.LATTICE_SHARED),
               dict(table_mode=P.TABLES_STAGED), dict(table_mode=P.TABLES_GLOBAL)):
        ok = P.Config(**{"L": 8, **kw}).to_c()
        assert lib.rewl_workspace_size(ctypes.byref(ok), ctypes.byref(n)) == 0


def test_product_path_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1508_02748_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
