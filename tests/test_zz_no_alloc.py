"""The no-allocation gate entry point, called through the C ABI.

tfhe_gate_batch_noalloc serves callers that cannot allocate device memory while they
run (their memory belongs to another allocator, or an allocation must not stall the
device mid-request); it keeps its scratch in a fixed array inside the library.  These
tests check, on two calls in a row, that it returns exactly what tfhe_gate_batch
returns (bit-exact, the tolerance of every parity test here), and that a batch too
big for the fixed scratch is refused before anything runs.  This file is collected
last so that a run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu


def call_noalloc(ctx, inp, types, idx, out, torch):
    import paper_2010_09410_b300 as tb
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return tb.lib().tfhe_gate_batch_noalloc(ctx.h, inp.data_ptr(), inp.shape[0],
                                            types.data_ptr(), idx.data_ptr(), out.data_ptr(),
                                            types.numel(), stream)


def test_noalloc_call_leaves_free_device_memory_unchanged(torch_cuda):
    """The context resolves the scratch array (and loads the entry point's kernels) when it
    is created, so not even the first call of the process allocates: free device memory
    (cudaMemGetInfo) is the same before and after it."""
    torch = torch_cuda
    params = ti.STD
    ctx, k = gpu_context(params, ti.SEED_FLAT)
    G = 64
    bits = ti.random_bits(ti.SEED_FLAT, 490, 2 * G)
    inp = to_dev(ti.encrypt_tlwe0_bits(params, ti.SEED_FLAT, 490, k.s0, bits))
    types = to_dev(ti.random_below(ti.SEED_FLAT, 491, G, 10).astype(np.uint8))
    idx = to_dev(np.arange(2 * G, dtype=np.int32).reshape(G, 2))
    got = torch.zeros((G, params.n + 1), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert call_noalloc(ctx, inp, types, idx, got, torch) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    ctx.sync()
    assert free1 == free0, (free0, free1)
    ref = torch.zeros_like(got)
    ctx.gate_batch(inp, types, idx, ref)
    ctx.sync()
    assert np.array_equal(from_dev(got), from_dev(ref))


@pytest.mark.parametrize("params,seed,sizes", [
    (ti.TOY, ti.SEED_TOY, (40, 23)),
    (ti.STD, ti.SEED_FLAT, (37, 195)),
])
def test_noalloc_matches_gate_batch_two_calls(torch_cuda, params, seed, sizes):
    torch = torch_cuda
    ctx, k = gpu_context(params, seed)
    for call, G in enumerate(sizes):
        bits = ti.random_bits(seed, 500 + call, 2 * G)
        b_inp = ti.encrypt_tlwe0_bits(params, seed, 500 + call, k.s0, bits)
        b_types = ti.random_below(seed, 600 + call, G, 10).astype(np.uint8)
        b_idx = np.arange(2 * G, dtype=np.int32).reshape(G, 2)
        inp, types, idx = to_dev(b_inp), to_dev(b_types), to_dev(b_idx)
        ref = torch.zeros((G, params.n + 1), dtype=torch.int32, device="cuda")
        got = torch.full((G, params.n + 1), -1, dtype=torch.int32, device="cuda")
        ctx.gate_batch(inp, types, idx, ref)
        assert call_noalloc(ctx, inp, types, idx, got, torch) == 0
        ctx.sync()
        assert np.array_equal(from_dev(got), from_dev(ref)), (call, G)
        import oracle as orc
        want = np.array([ti.plain_gate(t, bits[2 * g], bits[2 * g + 1])
                         for g, t in enumerate(b_types)], np.uint8)
        assert np.array_equal(orc.tlwe_decrypt(k.s0, from_dev(got)), want)


def test_noalloc_rejects_batches_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    ctx, k = gpu_context(ti.STD, ti.SEED_FLAT)
    G = 196
    inp = torch.zeros((2 * G, ti.STD.n + 1), dtype=torch.int32, device="cuda")
    types = torch.zeros(G, dtype=torch.uint8, device="cuda")
    idx = torch.zeros((G, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros((G, ti.STD.n + 1), dtype=torch.int32, device="cuda")
    assert call_noalloc(ctx, inp, types, idx, out, torch) == -1
    import paper_2010_09410_b300 as tb
    assert b"scratch" in tb.lib().tfhe_last_error(ctx.h)
    ctx.sync()
