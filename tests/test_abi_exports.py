"""The shared library loads and exports every entry point declared in
include/qtt.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qtt.h")
LIB = os.path.join(ROOT, "paper_2512_07811_gb300", "libqtt.so")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^QTT_API\s+[\w\s\*]+?\b(\w+)\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        sys.path.insert(0, ROOT)
        from paper_2512_07811_gb300 import build as B
        B.build(verbose=False)
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["tt_add", "tt_hadamard", "tt_mpo_apply", "tt_round", "tt_dot", "ms_homogenize",
                 "qtt_ctx_create", "qtt_tt_create", "qtt_status_string"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2512_07811_gb300 import qtt as Q
    assert sorted(Q.EXPORTED) == declared_symbols()


def test_status_strings_without_gpu(lib):
    lib.qtt_status_string.restype = ctypes.c_char_p
    assert lib.qtt_status_string(0) == b"ok"
    assert b"argument" in lib.qtt_status_string(-1)


def test_context_creation_fails_loudly_without_gpu(lib):
    """No device in this container: the context refuses instead of falling back."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    lib.qtt_ctx_create.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    st = lib.qtt_ctx_create(0, None, ctypes.byref(h))
    assert st != 0 and not h.value


def test_exports_are_c_symbols():
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    for s in declared_symbols():
        assert re.search(r"\sT\s%s$" % s, out, flags=re.M), s
