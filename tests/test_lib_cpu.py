"""CPU tests of the native library: it loads, exports every entry point that
include/hqr.h declares, and its host-side elimination-list generator and
validator agree with the oracle. No device work here."""
import itertools
import os
import re

import numpy as np
import pytest

from oracle.elim_list import BINARY, FIBONACCI, FLAT, GREEDY, TS, TT, hqr_elim_list, validate

hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    return hqr.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "hqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hqr_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(hqr.EXPORTS) == names


def test_strerror(lib):
    for code in range(8):
        assert lib.hqr_strerror(code)
    assert b"invalid" in lib.hqr_strerror(-3)


def test_lists_bit_exact_small(lib):
    trees = (FLAT, BINARY, GREEDY, FIBONACCI)
    for m in range(1, 8):
        for n in range(1, m + 1):
            for a in range(1, m + 1):
                for p in range(1, m + 1):
                    for lo, hi in itertools.product(trees, trees):
                        got = hqr.as_records(hqr.elim_list(m, n, a, p, lo, hi))
                        assert got == [tuple(r) for r in hqr_elim_list(m, n, a, p, lo, hi)]


@pytest.mark.parametrize("m,n,a,p", [(512, 8, 4, 16), (64, 64, 4, 1), (8, 8, 8, 1), (24, 10, 2, 3),
                                     (100, 37, 3, 7), (128, 16, 1, 1)])
def test_lists_bit_exact_workload_shapes(lib, m, n, a, p):
    for lo in (FLAT, BINARY, GREEDY, FIBONACCI):
        for hi in (FIBONACCI, GREEDY):
            got = hqr.elim_list(m, n, a, p, lo, hi)
            ref = hqr_elim_list(m, n, a, p, lo, hi)
            assert hqr.as_records(got) == [tuple(r) for r in ref]
            assert hqr.validate_list(m, n, got) == 0


def test_domino_lists_bit_exact(lib):
    trees = (FLAT, BINARY, GREEDY, FIBONACCI)
    for m in range(1, 8):
        for n in range(1, m + 1):
            for a in range(1, m + 1):
                for p in range(1, m + 1):
                    for lo, hi in itertools.product(trees, trees):
                        got = hqr.as_records(hqr.elim_list(m, n, a, p, lo, hi, domino=True))
                        assert got == [tuple(r) for r in hqr_elim_list(m, n, a, p, lo, hi, domino=True)]
    for (m, n, a, p) in [(24, 10, 2, 3), (512, 8, 4, 16), (100, 37, 3, 7)]:
        got = hqr.elim_list(m, n, a, p, GREEDY, FIBONACCI, domino=True)
        assert hqr.as_records(got) == [tuple(r) for r in hqr_elim_list(m, n, a, p, GREEDY, FIBONACCI, domino=True)]
        assert hqr.validate_list(m, n, got) == 0


def test_capacity_and_argument_errors(lib):
    import ctypes
    cnt = ctypes.c_size_t(0)
    assert lib.hqr_elim_list(8, 4, 2, 2, 0, 0, None, 0, ctypes.byref(cnt)) == hqr.ERR_CAPACITY
    assert cnt.value == 7 + 6 + 5 + 4
    assert lib.hqr_elim_list(0, 1, 1, 1, 0, 0, None, 0, ctypes.byref(cnt)) == -1
    assert lib.hqr_elim_list(4, 5, 1, 1, 0, 0, None, 0, ctypes.byref(cnt)) == -2
    assert lib.hqr_elim_list(4, 2, 0, 1, 0, 0, None, 0, ctypes.byref(cnt)) == -3
    assert lib.hqr_elim_list(4, 2, 1, 0, 0, 0, None, 0, ctypes.byref(cnt)) == -4
    assert lib.hqr_elim_list(4, 2, 1, 1, 7, 0, None, 0, ctypes.byref(cnt)) == -5
    assert lib.hqr_geqrf(None, 4, 4, 4, 0, 8, 4, None, 0, None, None) == -1
    # the widening entry point checks its arguments before any device work
    assert lib.hqr_widen_f32(None, None, -1, None) == -3
    assert lib.hqr_widen_f32(None, None, 0, None) == 0
    assert lib.hqr_widen_f32(None, ctypes.c_void_p(16), 4, None) == -1
    assert lib.hqr_widen_f32(ctypes.c_void_p(16), None, 4, None) == -2


def test_validator_agrees_with_oracle_on_mutations(lib):
    from tests.test_oracle_lists import _mutations
    L = hqr_elim_list(16, 4, 2, 2, BINARY, BINARY)
    assert hqr.validate_list(16, 4, L) == 0
    for name, M in _mutations(L):
        assert validate(M, 16, 4) is not None
        assert hqr.validate_list(16, 4, M) == hqr.ERR_INVALID_LIST, name
