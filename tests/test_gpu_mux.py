"""GPU HomMUX (Section 2.1.2 "Homomorphic Gates", "HomMUX without SE and IKS") against
the oracle: bit-exact TLWE and TRLWE outputs in both BlindRotate forms."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu

FORMS = [0, 1, 2, -1]
CASES = [(c, a, b) for c in (0, 1) for a in (0, 1) for b in (0, 1)]


def mux_inputs(p, seed, stream, k, cases):
    bits = np.array([x for case in cases for x in case], np.uint8)
    inp = ti.encrypt_tlwe0_bits(p, seed, stream, k.s0, bits)
    idx = np.arange(3 * len(cases), dtype=np.int32).reshape(len(cases), 3)
    return inp, idx


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("noks", [False, True])
def test_mux_toy_every_case_bit_exact(torch_cuda, form, noks):
    torch = torch_cuda
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    inp, idx = mux_inputs(p, ti.SEED_TOY, 41, k, CASES * 2)
    shape = (len(idx), 2, p.N) if noks else (len(idx), p.n + 1)
    out = torch.zeros(shape, dtype=torch.int32, device="cuda")
    ctx.mux_batch(to_dev(inp), to_dev(idx), out, form=form, noks=noks)
    ctx.sync()
    got = from_dev(out)
    want = orc.mux_batch(p, k.bsk, k.ksk, inp, idx, noks=noks)
    assert np.array_equal(got, want)
    if not noks:
        assert orc.tlwe_decrypt(k.s0, got).tolist() == [a if c else b for c, a, b in CASES * 2]


def test_mux_tfhe_like_batch(torch_cuda):
    """300 MUXes at n=630, N=1024: both forms give the same words, every output decrypts
    to c ? a : b, sampled MUXes match the oracle."""
    torch = torch_cuda
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_FLAT)
    G = 300
    bits = ti.random_bits(ti.SEED_FLAT, 42, 3 * G)
    inp = ti.encrypt_tlwe0_bits(p, ti.SEED_FLAT, 43, k.s0, bits)
    idx = np.arange(3 * G, dtype=np.int32).reshape(G, 3)
    outs = []
    for form in FORMS:
        out = torch.zeros((G, p.n + 1), dtype=torch.int32, device="cuda")
        ctx.mux_batch(to_dev(inp), to_dev(idx), out, form=form)
        ctx.sync()
        outs.append(from_dev(out))
    assert np.array_equal(outs[0], outs[1])
    b3 = bits.reshape(G, 3)
    want_bits = np.where(b3[:, 0] == 1, b3[:, 1], b3[:, 2])
    assert np.array_equal(orc.tlwe_decrypt(k.s0, outs[1]), want_bits)
    samples = [0, 151, G - 1]
    assert np.array_equal(outs[1][samples], orc.mux_batch(p, k.bsk, k.ksk, inp, idx, gates=samples))


def test_mux_bad_index_reported(torch_cuda):
    import paper_2010_09410_b300 as tb
    torch = torch_cuda
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    inp, idx = mux_inputs(p, ti.SEED_TOY, 44, k, CASES[:2])
    idx[1, 2] = 99
    out = torch.full((2, p.n + 1), -1, dtype=torch.int32, device="cuda")
    ctx.mux_batch(to_dev(inp), to_dev(idx), out)
    with pytest.raises(tb.TfheError):
        ctx.sync()
    got = from_dev(out)
    assert not got[1].any()
    want0 = orc.mux_batch(p, k.bsk, k.ksk, inp, idx[:1].copy())
    assert np.array_equal(got[0], want0[0])
