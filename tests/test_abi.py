"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/mpm.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mpm.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(mpm_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for need in ("mpm_octree_build", "mpm_assemble", "mpm_solve", "mpm_step", "mpm_create",
                 "mpm_destroy", "mpm_last_error"):
        assert need in syms


def test_library_exports_every_declared_symbol():
    from paper_2606_09275_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2606_09275_gb300 import mpm
    assert set(mpm.SYMBOLS) <= set(declared_symbols())
