"""The C-ABI library builds, loads and exports every entry point include/fe.h
declares (no GPU needed: nothing is called), and it carries none of the oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    text = open(os.path.join(ROOT, "include", "fe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*|int64_t)\s+(fe_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for need in ("fe_pattern", "fe_pattern_csr", "fe_pattern_slot_map", "fe_pattern_destroy",
                 "fe_assemble_mass", "fe_assemble_wmass", "fe_assemble_stiff", "fe_assemble_elas",
                 "fe_assemble_stiff_backward", "fe_batch_pattern", "fe_status"):
        assert need in names


def test_library_exports_every_declared_symbol():
    if not any(os.path.exists(os.path.join(p, "nvcc")) for p in os.environ.get("PATH", "").split(":")) \
            and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit to build the library")
    from paper_1401_3301_gb300 import build_ext
    path = build_ext.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.fe_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.fe_version()
    syms = subprocess.run(["nm", "-D", path], capture_output=True, text=True).stdout
    assert "orc_" not in syms  # the oracle is test infrastructure, never part of the library


def test_checked_library_exports_the_same_boundary():
    if not any(os.path.exists(os.path.join(p, "nvcc")) for p in os.environ.get("PATH", "").split(":")) \
            and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit to build the library")
    from paper_1401_3301_gb300 import build_ext
    path = build_ext.build(checked=True)
    assert path == build_ext.LIB_CHECKED
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.fe_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in lib.fe_version()
