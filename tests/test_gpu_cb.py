"""GPU circuit bootstrapping (Section 2.1.2 "Circuit Bootstrapping"; reading R16) against
the oracle: TRGSW words bit-exact, both steps separately, degenerate and ragged batches,
and, at N = 1024 / N2 = 2048, row phases, sampled words and CMUX-tree reads driven by
circuit-bootstrapped TLWE addresses."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu

_CB = {}


def cb_context(p, q, seed):
    """gpu_context with the circuit-bootstrapping keys of (p, q, seed) loaded."""
    import torch
    key = (p, q, seed)
    ctx, k = gpu_context(p, seed)
    if key not in _CB:
        cbk = ti.cb_keys(p, q, seed)
        bsk2 = torch.from_numpy(cbk.bsk2.view(np.int64)).cuda()
        pksk = to_dev(cbk.pksk)
        ctx.set_cb_keys(q, bsk2, pksk)
        ctx.sync()
        del bsk2, pksk
        _CB.clear()
        _CB[key] = cbk
    return ctx, k, _CB[key]


def run_cb(torch, ctx, p, tlwe):
    R = tlwe.shape[0]
    out = torch.zeros((R, 2 * p.l, 2, p.N), dtype=torch.int32, device="cuda")
    ctx.circuit_bootstrap(to_dev(tlwe), out)
    ctx.sync()
    return from_dev(out)


def run_tlwe2(torch, ctx, p, q, tlwe):
    R = tlwe.shape[0]
    out = torch.zeros((R, p.l, q.N2 + 1), dtype=torch.int64, device="cuda")
    ctx.cb_tlwe2(to_dev(tlwe), out)
    ctx.sync()
    return out.cpu().numpy().view(np.uint64)


def row_phase_errors(p, s1, trgsw, m):
    """Largest |phase - expected| (Torus32 units) over the 2l rows of a TRGSW of m."""
    s = s1.astype(np.int64)
    worst = 0
    for row in range(2 * p.l):
        g = 1 << (32 - (row % p.l + 1) * p.Bgbit)
        if row < p.l:
            expect = (-m * g * s) % 2**32
        else:
            expect = np.zeros(p.N, np.int64)
            expect[0] = m * g
        ph = orc.trlwe_phase(s1, trgsw[row]).astype(np.int64)
        err = ((ph - expect + 2**31) % 2**32) - 2**31
        worst = max(worst, int(np.abs(err).max()))
    return worst


# ---- toy parameters: every word --------------------------------------------------------

@pytest.mark.parametrize("R", [1, 5])
def test_circuit_bootstrap_toy_bit_exact(torch_cuda, R):
    p, q = ti.TOY, ti.CB_TOY
    ctx, k, cbk = cb_context(p, q, ti.SEED_CB)
    b = ti.cb_batch(p, q, ti.SEED_CB, R=R, stream=R)
    got = run_cb(torch_cuda, ctx, p, b.tlwe)
    want = orc.circuit_bootstrap(p, q, cbk.bsk2, cbk.pksk, b.tlwe)
    assert np.array_equal(got, want.reshape(got.shape))
    for r in range(R):
        assert row_phase_errors(p, k.s1, got[r], int(b.bits[r])) < 1 << 14


def test_cb_steps_toy_bit_exact(torch_cuda):
    """Step 1 (lvl2 TLWEs of m / Bg^u) and step 2 (private key switch, both functions)
    separately, each from the oracle's own inputs."""
    p, q = ti.TOY, ti.CB_TOY
    ctx, k, cbk = cb_context(p, q, ti.SEED_CB)
    b = ti.cb_batch(p, q, ti.SEED_CB, R=3, stream=11)
    t2 = run_tlwe2(torch_cuda, ctx, p, q, b.tlwe)
    for r in range(3):
        for u in range(1, p.l + 1):
            assert np.array_equal(t2[r, u - 1], orc.cb_tlwe2(p, q, cbk.bsk2, b.tlwe[r], u)), (r, u)
    rng = np.random.default_rng(5)
    J = 7
    src = rng.integers(0, 2**64, (J, q.N2 + 1), dtype=np.uint64)
    d_src = torch_cuda.from_numpy(src.view(np.int64)).cuda()
    for z in (0, 1):
        out = torch_cuda.zeros((J, 2, p.N), dtype=torch_cuda.int32, device="cuda")
        ctx.private_keyswitch(d_src, out, z)
        ctx.sync()
        got = from_dev(out)
        for j in range(J):
            assert np.array_equal(got[j], orc.private_keyswitch(p, q, cbk.pksk, z, src[j])), (z, j)


def test_circuit_bootstrap_degenerate_inputs(torch_cuda):
    """Trivial ciphertexts (all mask words 0: every BlindRotate step is the identity) with
    b at the ModSwitch edges, and mask words that all ModSwitch to 2 N2 - 1."""
    p, q = ti.TOY, ti.CB_TOY
    ctx, k, cbk = cb_context(p, q, ti.SEED_CB)
    rows = []
    for bval in (1 << 29, (-(1 << 29)) & 0xFFFFFFFF, 0, 0xFFFFFFFF, 1 << 31):
        c = np.zeros(p.n + 1, np.uint32)
        c[p.n] = bval
        rows.append(c)
    sh = 32 - (int(q.N2).bit_length())                  # 32 - log2(2 N2)
    c = np.full(p.n + 1, ((2 * q.N2 - 1) << sh) & 0xFFFFFFFF, np.uint32)
    assert orc.modswitch(q.N2, int(c[0])) == 2 * q.N2 - 1
    rows.append(c)
    tl = np.stack(rows)
    got = run_cb(torch_cuda, ctx, p, tl)
    want = orc.circuit_bootstrap(p, q, cbk.bsk2, cbk.pksk, tl)
    assert np.array_equal(got, want)
    assert row_phase_errors(p, k.s1, got[0], 1) < 1 << 14
    assert row_phase_errors(p, k.s1, got[1], 0) < 1 << 14


def test_circuit_bootstrap_errors(torch_cuda):
    import paper_2010_09410_b300 as tb
    p = ti.TOY
    ctx = tb.Context(p, 0)
    out = torch_cuda.zeros((1, 2 * p.l, 2, p.N), dtype=torch_cuda.int32, device="cuda")
    tl = torch_cuda.zeros((1, p.n + 1), dtype=torch_cuda.int32, device="cuda")
    with pytest.raises(tb.TfheError) as e:
        ctx.circuit_bootstrap(tl, out)
    assert e.value.code == -6  # ENOKEYS
    bad = ti.CBParams(N2=4096, l2=4, Bg2bit=9, pks_t=10, pks_basebit=3, sigma2=0.0,
                      sigma_pks=0.0)
    x = torch_cuda.zeros(16, dtype=torch_cuda.int64, device="cuda")
    with pytest.raises(tb.TfheError) as e:
        ctx.set_cb_keys(bad, x, x)
    assert e.value.code == -5  # EUNSUPPORTED
    ctx.close()
    ctx2, _, _ = cb_context(p, ti.CB_TOY, ti.SEED_CB)
    empty = torch_cuda.zeros((0, p.n + 1), dtype=torch_cuda.int32, device="cuda")
    ctx2.circuit_bootstrap(empty, out)  # R = 0 enqueues nothing
    ctx2.sync()


def test_cb_address_drives_cmux_tree_toy(torch_cuda):
    """TLWE address bits -> circuit bootstrapping -> CMUX-tree read, all on the GPU."""
    p, q = ti.TOY, ti.CB_TOY
    ctx, k, cbk = cb_context(p, q, ti.SEED_CB)
    rom = ti.cmux_rom(p, ti.SEED_CB, v=4, R=4, packed=p.N)
    bits = ((rom.addrs[:, None] >> np.arange(4)[None, :]) & 1).astype(np.uint8).reshape(-1)
    tl = ti.encrypt_tlwe0_bits(p, ti.SEED_CB, 96, k.s0, bits)
    addr = run_cb(torch_cuda, ctx, p, tl).reshape(4, 4, 2 * p.l, 2, p.N)
    out = torch_cuda.zeros((4, 2, p.N), dtype=torch_cuda.int32, device="cuda")
    ctx.cmux_tree_read(to_dev(addr), to_dev(rom.table), 4, out)
    ctx.sync()
    got = from_dev(out)
    for r in range(4):
        assert np.array_equal(orc.trlwe_decrypt(k.s1, got[r]), rom.table_bits[rom.addrs[r]])
        assert np.array_equal(got[r], orc.cmux_tree_read(p, addr[r], rom.table, 4))


# ---- N = 1024, N2 = 2048: the launch configuration of the benchmark --------------------------

def test_circuit_bootstrap_std_rows_and_samples(torch_cuda):
    """18 inputs (the address bits of two 9-bit reads, as the benchmark batches them):
    every TRGSW row decrypts within 2^18 of its message; step 2 word for word on two
    sampled lvl2 TLWEs; one lvl2 BlindRotate job word for word."""
    p, q = ti.STD, ti.CB_STD
    ctx, k, cbk = cb_context(p, q, ti.SEED_CB)
    b = ti.cb_batch(p, q, ti.SEED_CB, R=18, stream=12)
    got = run_cb(torch_cuda, ctx, p, b.tlwe)
    for r in range(18):
        assert row_phase_errors(p, k.s1, got[r], int(b.bits[r])) < 1 << 18, r
    t2 = run_tlwe2(torch_cuda, ctx, p, q, b.tlwe[:2])
    for r, u in ((0, 1), (1, 3)):
        ph = orc.tlwe2_phase(cbk.s2, t2[r, u - 1])
        expect = int(b.bits[r]) << (64 - u * p.Bgbit)
        d = (ph - expect) % 2**64
        assert min(d, 2**64 - d) < 1 << 44
        for z in (0, 1):
            want = orc.private_keyswitch(p, q, cbk.pksk, z, t2[r, u - 1])
            assert np.array_equal(got[r, z * p.l + u - 1], want), (r, u, z)
    assert np.array_equal(t2[1, 2], orc.cb_tlwe2(p, q, cbk.bsk2, b.tlwe[1], 3))


def test_cb_address_drives_cmux_tree_std(torch_cuda):
    """Two reads of the 512-row table with circuit-bootstrapped 9-bit addresses."""
    p, q = ti.STD, ti.CB_STD
    ctx, k, cbk = cb_context(p, q, ti.SEED_CB)
    rom = ti.cmux_rom(p, ti.SEED_CB, v=9, R=2)
    bits = ((rom.addrs[:, None] >> np.arange(9)[None, :]) & 1).astype(np.uint8).reshape(-1)
    tl = ti.encrypt_tlwe0_bits(p, ti.SEED_CB, 97, k.s0, bits)
    addr = run_cb(torch_cuda, ctx, p, tl).reshape(2, 9, 2 * p.l, 2, p.N)
    out = torch_cuda.zeros((2, 2, p.N), dtype=torch_cuda.int32, device="cuda")
    ctx.cmux_tree_read(to_dev(addr), to_dev(rom.table), 9, out)
    ctx.sync()
    got = from_dev(out)
    for r in range(2):
        assert np.array_equal(orc.trlwe_decrypt(k.s1, got[r]), rom.table_bits[rom.addrs[r]])
