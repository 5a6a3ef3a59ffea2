"""The CUDA library builds for sm_103a, loads without a GPU, and exports every
entry point that include/psi.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2601_05347_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(psi_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_last_error_without_gpu():
    lib = ctypes.CDLL(_build.build())
    lib.psi_last_error.restype = ctypes.c_char_p
    assert lib.psi_last_error() == b""
    lib.psi_launch_count.restype = ctypes.c_int64
    assert lib.psi_launch_count() >= 0
