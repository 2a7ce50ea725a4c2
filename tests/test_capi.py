"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/amg_gb300.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2202_09056_gb300 as amg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(amg_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("amg_setup", "amg_apply_vcycle", "amg_solve", "amg_free", "amg_bsr_spmv"):
        assert name in d


def test_library_exports_every_declared_symbol():
    lib = amg.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(amg.EXPORTED) <= _declared()


def test_build_targets_sm103a_only():
    from paper_2202_09056_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_default_params():
    p = amg.default_params()
    assert (p.eps_strong, p.relax, p.smooth_relax) == (0.08, 2.0, 0.8)
    assert (p.coarse_enough, p.max_levels, p.npre, p.npost, p.precision) == (3000, 15, 1, 1, 0)


def test_argument_errors_without_a_gpu():
    lib = amg.load()
    h = ctypes.c_void_p()
    assert lib.amg_setup(None, None, 6, None, None, ctypes.byref(h)) == -1
    assert lib.amg_last_error()
    A = amg.Bsr(4, 4, 3, 3, 0, None, None, None)
    assert lib.amg_setup(ctypes.byref(A), None, 6, None, None, ctypes.byref(h)) == -1
    assert lib.amg_solve(None, None, None, 1e-8, 10, None, None, None) == -1
    amg.load().amg_free(None)
