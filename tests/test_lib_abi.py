"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a,
loads, exports every function the public header declares, and rejects bad
arguments before touching a device."""
import ctypes
import os
import re

import pytest

import paper_2010_09410_b300 as tb
from paper_2010_09410_b300 import build as tbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tfhe_b300.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tfhe_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    tbuild.build()
    return tb.lib()


def test_header_and_binding_agree():
    assert header_functions() == sorted(tb.EXPORTS)


def test_library_exports_every_header_symbol(L):
    for name in header_functions():
        assert hasattr(L, name), name
    assert L.tfhe_version() == 10000


def test_null_arguments_rejected_without_device(L):
    out = ctypes.c_void_p()
    assert L.tfhe_ctx_create(None, 0, ctypes.byref(out)) == -1
    p = tb.CParams(630, 1024, 3, 6, 8, 2)
    assert L.tfhe_ctx_create(ctypes.byref(p), 0, None) == -1
    assert L.tfhe_gate_batch(None, None, 0, None, None, None, 1, 0, None) == -1
    assert L.tfhe_cmux_tree_read(None, None, None, 9, None, 1, 0, None) == -1
    assert L.tfhe_plan_run(None, None, None, 0, None, None) == -1
    assert L.tfhe_plan_num_levels(None) == -1
    buf = ctypes.create_string_buffer(b"x" * 8)
    assert L.tfhe_last_error_string(None, buf, 8) == -1 and buf.value == b""
    assert L.tfhe_last_error_string(None, None, 0) == -1
    L.tfhe_ctx_destroy(None)
    L.tfhe_plan_destroy(None)


@pytest.mark.parametrize("bad", [
    (630, 1000, 3, 6, 8, 2),   # N not a power of two
    (630, 4096, 3, 6, 8, 2),   # N too large
    (630, 1024, 6, 6, 8, 2),   # l * Bgbit > 31
    (0, 1024, 3, 6, 8, 2),     # n < 1
    (630, 1024, 3, 6, 16, 2),  # t * basebit > 31
])
def test_unsupported_parameters_rejected(L, bad):
    out = ctypes.c_void_p()
    assert L.tfhe_ctx_create(ctypes.byref(tb.CParams(*bad)), 0, ctypes.byref(out)) == -5
