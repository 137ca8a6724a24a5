"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in include/dgpmg.h.

No compute call is made here (no GPU is needed)."""
import ctypes
import os
import re

import pytest

import paper_1809_00866_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dgpmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_matches_binding_exports():
    assert declared_symbols() == sorted(P.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = P.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_create_rejects_bad_params_without_gpu_work():
    # argument checks run before any CUDA call
    L = P.load()
    h = ctypes.c_void_p()
    params = P.DgParams()
    params.nx = 1
    assert L.dg_create(ctypes.byref(params), ctypes.byref(h)) == P.DG_ERR_ARG
    assert b"at least 2 cells" in L.dg_last_error(None)
    assert L.dg_create(None, ctypes.byref(h)) == P.DG_ERR_ARG
