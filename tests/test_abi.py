"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/icnnm.h declares (no compute calls here)."""
import ctypes as C
import os
import re

import pytest

from paper_2604_17001_gb300 import icnnm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "icnnm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(icnnm_[a-zA-Z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(icnnm.LIB_PATH):
        from paper_2604_17001_gb300 import build
        build.build()
    return icnnm.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["icnnm_learn_V", "icnnm_solve", "icnnm_submit", "icnnm_poll", "icnnm_create", "icnnm_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_status_strings_and_defaults(lib):
    for st in range(10):
        assert lib.icnnm_strerror(st)
    p = icnnm.icnnm_params()
    assert lib.icnnm_params_default(C.byref(p)) == 0
    assert p.lambda_ == float("inf") and p.rho == 1.1 and p.theta_max == 1e10 and p.max_iters == 100
    assert lib.icnnm_params_default(None) == icnnm.EINVAL


def test_null_arguments_are_errors_not_crashes(lib):
    assert lib.icnnm_create(None, 0, 0, None) == icnnm.EINVAL
    assert lib.icnnm_solve(None, None, None, None, None, None, None, None) == icnnm.EINVAL
    assert lib.icnnm_poll(None, 1, None, None) == icnnm.EINVAL
    assert lib.icnnm_learn_V(None, None, 0, None, None, None, None) == icnnm.EINVAL
    assert lib.icnnm_cnnm_solve(None, None, None, None, None, None, None) == icnnm.EINVAL
    assert lib.icnnm_spectral_diagnostics(None, None, None, None, 1e-6, None, None, None, None) == icnnm.EINVAL
    lib.icnnm_destroy(None)
    assert lib.icnnm_last_error(None) == b""
