"""Failure detection without a GPU fault: a bounded device wait on a flag that nothing
sets gives up, records TFHE_ETIMEOUT in the context's device error word, tfhe_ctx_sync
reports and clears it, and the context keeps working (bit-exact gates afterwards)."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu


def test_wait_timeout_reported_and_context_usable(torch_cuda):
    import paper_2010_09410_b300 as tb
    torch = torch_cuda
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")  # nothing ever sets it
    ctx.probe_wait(flag, 1, 200_000_000)                      # about 0.1 s of SM clocks
    with pytest.raises(tb.TfheError) as e:
        ctx.sync()
    assert e.value.code == -4  # TFHE_ETIMEOUT
    ctx.sync()                 # the error word was cleared
    b = ti.toy_gates()
    out = torch.zeros((b.types.size, p.n + 1), dtype=torch.int32, device="cuda")
    ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=0)
    ctx.sync()
    assert np.array_equal(from_dev(out), orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx))


def test_wait_on_a_set_flag_returns(torch_cuda):
    torch = torch_cuda
    ctx, _ = gpu_context(ti.TOY, ti.SEED_TOY)
    flag = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    ctx.probe_wait(flag, 3, 200_000_000)
    ctx.sync()


def test_wait_arguments_checked_on_host(torch_cuda):
    import paper_2010_09410_b300 as tb
    torch = torch_cuda
    ctx, _ = gpu_context(ti.TOY, ti.SEED_TOY)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    for bad in (-1, 9_000_000_000):
        with pytest.raises(tb.TfheError) as e:
            ctx.probe_wait(flag, 1, bad)
        assert e.value.code == -1
    ctx.sync()


def test_last_error_string_copies_and_truncates(torch_cuda):
    """tfhe_last_error_string copies the context's last error text (the same text
    tfhe_last_error returns), NUL-terminated, truncated to the buffer, and returns the
    text's full length."""
    import ctypes
    import paper_2010_09410_b300 as tb
    ctx, _ = gpu_context(ti.STD, ti.SEED_FLAT)
    with pytest.raises(tb.TfheError):
        ctx.set_tc_pass_limit((1 << 17) + 1)
    L = tb.lib()
    text = L.tfhe_last_error(ctx.h)
    assert text
    big = ctypes.create_string_buffer(len(text) + 16)
    assert L.tfhe_last_error_string(ctx.h, big, len(big)) == len(text)
    assert big.value == text
    small = ctypes.create_string_buffer(b"#" * 8)
    assert L.tfhe_last_error_string(ctx.h, small, 8) == len(text)
    assert small.value == text[:7]
    assert L.tfhe_last_error_string(ctx.h, None, 0) == len(text)
