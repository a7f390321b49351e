"""The C-ABI library loads and exports every entry point include/nqs.h
declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nqs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nqs_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("nqs_sample", "nqs_logpsi", "nqs_local_energy", "nqs_jacobian", "nqs_minsr_step"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2608_18065_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    lib.nqs_status_string.restype = ctypes.c_char_p
    assert lib.nqs_status_string(5) == b"T + lambda I not positive definite"
