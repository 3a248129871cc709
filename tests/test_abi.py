"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/qe.h declares, the Python binding covers exactly
those, and argument validation that happens before any device work returns
the documented status codes."""
import ctypes as C
import re
from pathlib import Path

import pytest

from paper_1604_06460_gb300 import build as B
from paper_1604_06460_gb300 import qe

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        names |= set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(qe_\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return qe.load()


def test_header_declares_core_entry_points():
    names = declared_functions()
    for core in ["qe_alloc_state", "qe_free_state", "qe_apply_gate", "qe_apply_qft",
                 "qe_apply_add_const", "qe_expectation", "qe_probs", "qe_flush",
                 "qe_sync", "qe_last_error"]:
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_matches_header():
    assert set(qe.SIGNATURES) == declared_functions()


def test_argument_errors_before_device_work(lib):
    h = C.c_void_p()
    assert lib.qe_alloc_state(0, qe.C128, None, 0, None, C.byref(h)) == -1
    assert b"n must be" in lib.qe_last_error()
    assert lib.qe_alloc_state(40, qe.C128, None, 0, None, C.byref(h)) == -1
    assert lib.qe_alloc_state(4, 7, None, 0, None, C.byref(h)) == -1
    assert lib.qe_alloc_state(4, qe.C128, None, 0, None, None) == -1
    # a borrowed buffer that is too small is rejected before it is touched
    assert lib.qe_alloc_state(4, qe.C128, C.c_void_p(256), 16, None, C.byref(h)) == -1
    assert b"too small" in lib.qe_last_error()
    # misaligned borrowed buffer
    assert lib.qe_alloc_state(4, qe.C128, C.c_void_p(8), 1 << 20, None, C.byref(h)) == -1
    assert b"aligned" in lib.qe_last_error()


def test_null_and_invalid_handles(lib):
    assert lib.qe_free_state(None) == 0
    assert lib.qe_flush(None) == -5
    assert lib.qe_apply_qft(None, 0, 1, 0) == -5
    bogus = (C.c_char * 4096)()
    assert lib.qe_sync(C.cast(bogus, C.c_void_p)) == -5
