import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Rows of a whitespace-separated golden fixture, comments stripped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def pins_lib():
    """The exhaustive C checkers of tests/pins_exhaustive.c, compiled on first use."""
    import ctypes
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "pins_exhaustive.c")
    so = os.path.join(here, "libpins_exhaustive.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", so, src])
    lib = ctypes.CDLL(so)
    u64, vp, i32 = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
    lib.chk_decompose.argtypes = [vp, i32, i32, u64, u64]
    lib.chk_ks_digits.argtypes = [vp, i32, i32, u64, u64]
    lib.chk_modswitch.argtypes = [vp, i32, u64, u64]
    for f in (lib.chk_decompose, lib.chk_ks_digits, lib.chk_modswitch):
        f.restype = u64
    return lib
