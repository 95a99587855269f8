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


# ---- GPU fixtures ------------------------------------------------------------------

def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="session")
def torch_cuda():
    return _cuda()


_CTX = {}


def gpu_context(params, seed):
    """A library context on cuda:0 with the seeded keys of (params, seed) loaded."""
    key = (params, seed)
    if key not in _CTX:
        torch = _cuda()
        import paper_2010_09410_b300 as tb
        import tfhe_inputs as ti
        from paper_2010_09410_b300 import build as tbuild
        tbuild.build()
        k = ti.keys(params, seed)
        ctx = tb.Context(params, 0)
        bsk = torch.from_numpy(k.bsk.view("int32")).cuda()
        ksk = torch.from_numpy(k.ksk.view("int32")).cuda()
        ctx.set_keys(bsk, ksk)
        ctx.sync()
        _CTX[key] = (ctx, k)
    return _CTX[key]


def to_dev(a):
    """numpy uint32/uint8/int32 array -> CUDA tensor with the same bytes."""
    import numpy as np
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def from_dev(t):
    """CUDA int32 tensor -> numpy uint32."""
    import numpy as np
    return t.cpu().numpy().view(np.uint32)
