"""The C-ABI library loads and exports every entry point that include/pff.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pff.h")
LIB = os.path.join(ROOT, "paper_2203_16467_gb300", "libpff.so")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pff_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpff():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pff_create_problem", "pff_set_modulus_field", "pff_set_model", "pff_step_load", "pff_get_fields",
                 "pff_create_batch", "pff_batch_admit", "pff_batch_step", "pff_batch_release"):
        assert must in names


def test_library_exports_every_declared_symbol(libpff):
    missing = [n for n in declared_functions() if not hasattr(libpff, n)]
    assert not missing, missing


def test_binding_loads_and_defaults_match_paper(libpff):
    from paper_2203_16467_gb300 import pff
    p = pff.default_params()
    assert p.nu == 0.2 and p.mech_tol == 1e-6 and p.pf_tol == 1e-6 and p.dphi_min == 1e-3
    assert p.crack_set_threshold == 0.9
    assert pff.problem_bytes(64, 64, pff.MIXED) < pff.problem_bytes(64, 64, pff.FP64)


def test_invalid_sizes_rejected_without_gpu(libpff):
    from paper_2203_16467_gb300 import pff
    h = ctypes.c_void_p()
    assert pff.lib.pff_create_problem(48, 64, pff.MIXED, None, ctypes.byref(h)) == pff.ERR_INVALID_ARG
    assert pff.lib.pff_create_problem(64, 64, 7, None, ctypes.byref(h)) == pff.ERR_INVALID_ARG


def test_kernel_variant_arguments_checked_without_gpu(libpff):
    from paper_2203_16467_gb300 import pff
    assert pff.lib.pff_set_kernel_variant(0, 512, 1, 1) == pff.ERR_INVALID_ARG
    assert pff.lib.pff_set_kernel_variant(pff.VARIANT_COLUMN_SHAPE, 512, 2, 0) == pff.ERR_INVALID_ARG
    assert pff.lib.pff_set_kernel_variant(pff.VARIANT_COLUMN_SHAPE, 512, 1, 2) == pff.ERR_INVALID_ARG
    assert pff.lib.pff_set_kernel_variant(pff.VARIANT_BCCG_PASSES, 0, 1, -1) == pff.ERR_INVALID_ARG
    assert pff.lib.pff_set_barrier_spin_limit(-1) == pff.ERR_INVALID_ARG
