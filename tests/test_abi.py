"""The C-ABI library loads without a GPU and exports every entry point that
include/pgk.h declares; host-only calls behave (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1801_04348_gb300 import build as pbuild
from paper_1801_04348_gb300 import pgk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pbuild.build()
    return pgk.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "pgk.h")).read()
    return sorted(set(re.findall(r"^PGK_API\s+[\w\s\*]+?\b(pgk_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = header_functions()
    for must in ("pgk_gemm", "pgk_gemm_grouped", "pgk_select_case", "pgk_machine_query"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    for name in header_functions():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_binding_covers_header():
    assert sorted(pgk.symbols()) == header_functions()


def test_status_strings_and_version(L):
    assert L.pgk_abi_version() == 1
    for code, name in pgk.STATUS.items():
        assert L.pgk_status_string(code).decode() == name


def test_variant_registry_without_gpu(L):
    n = pgk.num_variants()
    assert n >= 10
    fams = [pgk.variant_info_get(i).family for i in range(n)]
    assert pgk.FAM_PAPER in fams and pgk.FAM_RB in fams and pgk.FAM_DIRECT in fams


def test_invalid_arguments_are_errors_not_crashes(L):
    m = pgk.Machine(1024, 49152, 232448, 65536, 65536, 255, 2048, 152, 32, 10, 3, 0)
    regs = [32] * pgk.REG_CLASSES
    st, _ = pgk.select_case_regs(m, regs, 0, 16, 16, pgk.F32, pgk.params(16, 16, 2))
    assert st == 1  # INVALID_ARG: zero size
    st, _ = pgk.select_case_regs(m, regs, 16, 16, 16, pgk.F32, pgk.params(0, 16, 2))
    assert st == 1
    st, _ = pgk.select_case_regs(m, regs, 16, 16, 16, pgk.F32, pgk.params(32, 8, 2))
    assert st == 2  # INFEASIBLE: B0 <= B1*s fails
    st, _ = pgk.select_case_regs(m, regs, 16, 16, 16, pgk.F32, pgk.params(16, 16, 3, 3, 8))
    assert st == 3  # UNSUPPORTED: no such register-blocked variant
    assert L.pgk_gemm(0, 1, 1, 0, None, 1, None, 1, None, 1, 0, None, None) == 1
    assert L.pgk_cvt_bf16(0, 1, None, 1, None, 1, 0, None) == 1
    assert L.pgk_simt_peak_probe(0, 1, 1, None, None) == 1
    assert L.pgk_gemm_host(0, 1, 1, 0, None, 1, None, 1, None, 1, 0, None, None) == 1
