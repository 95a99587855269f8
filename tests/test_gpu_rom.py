"""GPU ROM with vertical and horizontal packing (Section 8.3) against the oracle."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu


def read(torch, ctx, p, rom):
    R = rom.addr_trgsw.shape[0]
    trlwe = torch.zeros((R, 2, p.N), dtype=torch.int32, device="cuda")
    bits = torch.zeros((R, rom.w, p.n + 1), dtype=torch.int32, device="cuda")
    ctx.rom_read(to_dev(rom.addr_trgsw), to_dev(rom.table), rom.v, rom.w, trlwe, bits)
    ctx.sync()
    return from_dev(trlwe), from_dev(bits)


@pytest.mark.parametrize("M,w", [(32, 32), (32, 8), (8, 64)])
def test_packed_rom_toy_every_address_bit_exact(torch_cuda, M, w):
    """Every address of toy ROMs (several TRLWEs, one TRLWE with a tree of zero levels)."""
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    rom = ti.packed_rom(p, ti.SEED_TOY, M=M, w=w, R=M, stream=7)
    rom.addrs[:] = np.arange(M)
    abits = ((rom.addrs[:, None] >> np.arange(rom.v)[None, :]) & 1).astype(np.uint8)
    rom.addr_trgsw = ti.encrypt_trgsw_bits(p, ti.SEED_TOY, 90, k.s1, abits.reshape(-1)).reshape(
        M, rom.v, 2 * p.l, 2, p.N)
    trlwe, bits = read(torch_cuda, ctx, p, rom)
    for r in range(M):
        want_t, want_b = orc.rom_read(p, k.ksk, rom.addr_trgsw[r], rom.table, rom.v, rom.w)
        assert np.array_equal(trlwe[r], want_t), r
        assert np.array_equal(bits[r], want_b), r
        assert np.array_equal(orc.tlwe_decrypt(k.s0, bits[r]), rom.words[r]), r


def test_paper_rom_512_bytes(torch_cuda):
    """The paper's ROM: 128 words of 32 bits in 4 TRLWEs at N = 1024, 16 reads: every
    read decrypts to its word, sampled reads match the oracle word for word."""
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_CMUX)
    rom = ti.packed_rom(p, ti.SEED_CMUX, M=128, w=32, R=16, stream=8)
    trlwe, bits = read(torch_cuda, ctx, p, rom)
    for r in range(16):
        assert np.array_equal(orc.tlwe_decrypt(k.s0, bits[r]), rom.words[rom.addrs[r]]), r
    for r in (0, 15):
        want_t, want_b = orc.rom_read(p, k.ksk, rom.addr_trgsw[r], rom.table, rom.v, rom.w)
        assert np.array_equal(trlwe[r], want_t) and np.array_equal(bits[r], want_b), r
