"""The C-ABI library loads and exports every entry point the header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tcng.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tcng_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_14167_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_core_calls():
    names = declared()
    for n in ["tcng_state_init", "tcng_apply_circuit", "tcng_expect_pauli", "tcng_energy_grad"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_2602_14167_b300 import tcng
    assert set(declared()) <= set(tcng.EXPORTED)


def test_version_and_error_calls_need_no_gpu(lib):
    lib.tcng_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.tcng_version()
    lib.tcng_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.tcng_last_error(), bytes)
