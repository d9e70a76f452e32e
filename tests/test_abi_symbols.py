"""The C-ABI library loads and exports every entry point that include/qs.h
declares; host-side argument validation answers without touching a GPU.
CPU only (no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qs.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import build
    if not os.path.exists(build.LIB_PATH):
        build.build()
    from paper_2311_01512_gb300 import qs as mod
    return mod


def test_header_declares_the_hot_path(qs):
    names = declared_symbols()
    for required in ("qs_create_statevector", "qs_create_densmatr", "qs_apply_ctrl_multi_target",
                     "qs_apply_pauli_gadget", "qs_apply_kraus", "qs_partial_trace", "qs_expec_pauli_sum"):
        assert required in names


def test_library_exports_every_declared_symbol(qs):
    lib = ctypes.CDLL(qs.lib_path())
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert missing == []
    # and the binding knows every one of them
    assert sorted(qs.SIGNATURES) == declared_symbols()


def test_host_validation_without_gpu(qs):
    lib = ctypes.CDLL(qs.lib_path())
    lib.qs_create_statevector.restype = ctypes.c_int
    h = ctypes.c_void_p()
    # null device pointer
    assert lib.qs_create_statevector(4, 1, None, None, ctypes.byref(h)) == 1
    # unaligned device pointer is rejected before any CUDA call
    assert lib.qs_create_statevector(4, 1, ctypes.c_void_p(0x1008), None, ctypes.byref(h)) == 10
    # bad precision, too many storage qubits
    assert lib.qs_create_statevector(4, 7, ctypes.c_void_p(0x1000), None, ctypes.byref(h)) == 1
    assert lib.qs_create_densmatr(18, 1, ctypes.c_void_p(0x1000), None, ctypes.byref(h)) == 1
    # null handles
    assert lib.qs_apply_dephasing(None, 0, ctypes.c_double(0.1)) == 1
    lib.qs_status_str.restype = ctypes.c_char_p
    assert lib.qs_status_str(4) == b"qubit is both target and control"
