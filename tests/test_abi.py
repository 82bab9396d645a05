"""The C-ABI library loads and exports every entry point declared in include/qnep.h.

CPU only: no call touches a GPU (qnep_param_count and qnep_status_string are
pure host functions).
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2601_19034_gb300 import _lib
from paper_2601_19034_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "qnep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qnep_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert "qnep_compute" in names and "qnep_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_param_count_matches_documented_layout(lib):
    for s in (1, 2, 3, 4):
        hp = wl.HParams(n_species=s)
        c = _lib.HParamsC(hp.n_species, hp.rc_radial, hp.rc_angular, hp.n_radial, hp.n_angular,
                          hp.basis_radial, hp.basis_angular, hp.l_max, hp.use_4body, hp.n_neurons)
        assert lib.qnep_param_count(ctypes.byref(c)) == hp.n_params


def test_status_strings(lib):
    for code in range(7):
        assert lib.qnep_status_string(code)
    assert lib.qnep_status_string(_lib.QNEP_ERR_NBR_OVERFLOW).decode() == "neighbour list overflow"


def test_struct_layouts_match_header():
    # qnep_elec: int, int, double x3, int[3], int, double -> 56 bytes with natural alignment
    assert ctypes.sizeof(_lib.ElecC) == 56
    assert ctypes.sizeof(_lib.HParamsC) == 40
    assert ctypes.sizeof(_lib.OutputsC) == 64
