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


def test_binding_refuses_host_or_missized_buffers_before_the_call():
    # the library cannot see a device buffer's size or type: the binding checks
    # every tensor it hands over (no GPU needed, nothing reaches the library)
    import numpy as np
    import pytest
    import torch
    from paper_2606_09275_gb300 import mpm
    for bad in (torch.zeros(6, dtype=torch.float64), np.zeros(6),
                torch.zeros(6, dtype=torch.float32), torch.zeros(12, dtype=torch.float64)[::2]):
        with pytest.raises(mpm.MPMError) as e:
            mpm._check_vec("solve", "rhs", bad, torch.float64, 6)
        assert e.value.code == 1 and "rhs" in str(e.value)
    assert mpm._k_dtype(mpm.MIXED) == torch.float32 and mpm._k_dtype(mpm.FP64) == torch.float64
    with pytest.raises(mpm.MPMError):
        mpm._check_vec("step", "du_out", torch.zeros(6, dtype=torch.float32), torch.float64)
