"""Other ring degrees: N = 512 (three radix-8 passes per transform, Karatsuba level 1 in
the tensor-core form) and N = 2048 (passes of 3, 3, 3, 2; no tensor-core form).  Gates
in every supported form and CMUX batches, word for word against the oracle."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu

P512 = ti.Params(n=100, N=512, l=3, Bgbit=6, ks_t=8, ks_basebit=2, sigma0=2.0**-15,
                 sigma1=2.0**-25)
P2048 = ti.Params(n=16, N=2048, l=3, Bgbit=6, ks_t=8, ks_basebit=2, sigma0=2.0**-15,
                  sigma1=2.0**-25)
SEED = 0x20100941 + 40


@pytest.mark.parametrize("p,G", [(P512, 12), (P2048, 6)])
def test_gates_every_form(torch_cuda, p, G):
    import paper_2010_09410_b300 as tb
    torch = torch_cuda
    ctx, k = gpu_context(p, SEED)
    b = ti.flat_level(G, seed=SEED, p=p)
    want = orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx)
    assert np.array_equal(orc.tlwe_decrypt(k.s0, want), b.expected)
    for form in (0, 2, 1, -1):
        out = torch.zeros((G, p.n + 1), dtype=torch.int32, device="cuda")
        if form == 1 and p.N > 1024:
            with pytest.raises(tb.TfheError) as e:
                ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
            assert e.value.code == -5  # EUNSUPPORTED
            continue
        ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
        ctx.sync()
        assert np.array_equal(from_dev(out), want), form


@pytest.mark.parametrize("p", [P512, P2048])
def test_cmux_batch(torch_cuda, p):
    ctx, k = gpu_context(p, SEED)
    rng = np.random.default_rng(p.N)
    B, group = 5, 2
    ny = (B + group - 1) // group
    sel = ti.encrypt_trgsw_bits(p, 7, 1, k.s1, rng.integers(0, 2, ny).astype(np.uint8))
    d1 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
    d0 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
    out = to_dev(np.zeros_like(d0))
    ctx.cmux_batch(to_dev(sel), group, to_dev(d1), to_dev(d0), out, form=0)
    ctx.sync()
    got = from_dev(out)
    for q in range(B):
        assert np.array_equal(got[q], orc.cmux(p, sel[q // group], d1[q], d0[q])), q


def test_tc_levels_at_n512(torch_cuda):
    """The tensor-core form at N = 512 on every Karatsuba level it supports (level 0: 4
    stages of 128 digits per row; level 2: s = 128, one stage), 140 gates (a full tile and a
    ragged one), word for word against the oracle on the first and last gate of each tile."""
    torch = torch_cuda
    p = P512
    ctx, k = gpu_context(p, SEED)
    G = 140
    b = ti.flat_level(G, seed=SEED, p=p)
    sample = [0, 127, 128, 139]
    want = orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx, gates=sample)
    try:
        for level in (0, 1, 2):
            ctx.set_tc_level(level)
            out = torch.zeros((G, p.n + 1), dtype=torch.int32, device="cuda")
            ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=1)
            ctx.sync()
            got = from_dev(out)
            assert np.array_equal(orc.tlwe_decrypt(k.s0, got), b.expected), level
            assert np.array_equal(got[sample], want), level
    finally:
        ctx.set_tc_level(-1)
