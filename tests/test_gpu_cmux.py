"""GPU parity of the CMUX Memory units (Section 8.2) against the CPU oracle."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu

FORMS = [0, 2, 1]  # form 1 (tensor cores) covers groups of >= 128 CMUXes per selector


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("B,group", [(7, 3), (16, 16), (5, 1)])
def test_cmux_batch_toy(torch_cuda, form, B, group):
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    rng = np.random.default_rng(B * 10 + group)
    ny = (B + group - 1) // group
    sel = ti.encrypt_trgsw_bits(p, 5, 1, k.s1, rng.integers(0, 2, ny).astype(np.uint8))
    d1 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
    d0 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
    out = to_dev(np.zeros_like(d0))
    ctx.cmux_batch(to_dev(sel), group, to_dev(d1), to_dev(d0), out, form=form)
    ctx.sync()
    got = from_dev(out)
    for q in range(B):
        assert np.array_equal(got[q], orc.cmux(p, sel[q // group], d1[q], d0[q])), q


@pytest.mark.parametrize("form", FORMS)
def test_cmux_tree_read_toy_every_address(torch_cuda, form):
    p = ti.TOY
    rom = ti.cmux_rom(p, ti.SEED_TOY, v=4, R=16, packed=p.N)
    ctx, k = gpu_context(p, ti.SEED_TOY)
    out = to_dev(np.zeros((16, 2, p.N), np.uint32))
    ctx.cmux_tree_read(to_dev(rom.addr_trgsw), to_dev(rom.table), 4, out, form=form)
    ctx.sync()
    got = from_dev(out)
    for r in range(16):
        assert np.array_equal(got[r], orc.cmux_tree_read(p, rom.addr_trgsw[r], rom.table, 4)), r
        assert np.array_equal(orc.trlwe_decrypt(k.s1, got[r]), rom.table_bits[rom.addrs[r]])


_TREE_WANT = {}


def tree_read_sample(rom):
    """Eight of the 64 reads (the first, the last and six seeded others) with the oracle's
    words, computed once (in threads: the C oracle releases the interpreter lock)."""
    if not _TREE_WANT:
        from concurrent.futures import ThreadPoolExecutor
        reads = sorted({0, 63} | set(int(r) for r in
                                     np.random.default_rng(11).choice(np.arange(1, 63), 6, replace=False)))
        with ThreadPoolExecutor(len(reads)) as ex:
            want = list(ex.map(lambda r: orc.cmux_tree_read(ti.STD, rom.addr_trgsw[r], rom.table, 9),
                               reads))
        _TREE_WANT.update(zip(reads, want))
    return _TREE_WANT


@pytest.mark.parametrize("form", FORMS)
def test_cmux_tree_read_512_rows_64_reads(torch_cuda, form):
    """512-row table, 9 address bits, 64 reads: all reads decrypt to the addressed row,
    eight reads match the oracle word for word."""
    p = ti.STD
    rom = ti.cmux_rom()
    ctx, k = gpu_context(p, ti.SEED_CMUX)
    out = to_dev(np.zeros((64, 2, p.N), np.uint32))
    ctx.cmux_tree_read(to_dev(rom.addr_trgsw), to_dev(rom.table), 9, out, form=form)
    ctx.sync()
    got = from_dev(out)
    for r in range(64):
        assert np.array_equal(orc.trlwe_decrypt(k.s1, got[r])[:32], rom.table_bits[rom.addrs[r], :32])
    want = tree_read_sample(rom)
    assert len(want) == 8
    for r, w in want.items():
        assert np.array_equal(got[r], w), r


@pytest.mark.parametrize("B,group", [(256, 128), (300, 150), (700, 700), (350, 150)])
def test_cmux_batch_tensor_cores_toy(torch_cuda, B, group):
    """Tensor-core CMUX batches: one or several 128-CMUX tiles per selector, with ragged
    groups (150 = 128 + 22 padding rows; 700 over six tiles; 350 = two groups of 150 and
    a last group of 50), every CMUX word for word against the oracle and the NTT form."""
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    rng = np.random.default_rng(B + group)
    ny = (B + group - 1) // group
    sel = ti.encrypt_trgsw_bits(p, 7, 3, k.s1, rng.integers(0, 2, ny).astype(np.uint8))
    d1 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
    d0 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
    outs = {}
    for form in (1, 2):
        out = to_dev(np.zeros_like(d0))
        ctx.cmux_batch(to_dev(sel), group, to_dev(d1), to_dev(d0), out, form=form)
        ctx.sync()
        outs[form] = from_dev(out)
    assert np.array_equal(outs[1], outs[2])
    for q in range(B):
        assert np.array_equal(outs[1][q], orc.cmux(p, sel[q // group], d1[q], d0[q])), q


def test_cmux_tree_read_tensor_cores_toy(torch_cuda):
    """A 256-row toy table (8 address bits): tree level 0 has 128 CMUXes per read and runs
    on the tensor cores, the other levels in the NTT form; both reads word for word."""
    p = ti.TOY
    rom = ti.cmux_rom(p, ti.SEED_TOY, v=8, R=2, packed=32)
    ctx, k = gpu_context(p, ti.SEED_TOY)
    out = to_dev(np.zeros((2, 2, p.N), np.uint32))
    ctx.cmux_tree_read(to_dev(rom.addr_trgsw), to_dev(rom.table), 8, out, form=1)
    ctx.sync()
    got = from_dev(out)
    for r in range(2):
        assert np.array_equal(got[r], orc.cmux_tree_read(p, rom.addr_trgsw[r], rom.table, 8)), r
        assert np.array_equal(orc.trlwe_decrypt(k.s1, got[r])[:32], rom.table_bits[rom.addrs[r], :32])


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("v", [1, 3])
def test_ram_write_toy(torch_cuda, form, v):
    p = ti.TOY
    ram = ti.ram_write(p, ti.SEED_TOY, v=v, packed=p.N)
    ctx, k = gpu_context(p, ti.SEED_TOY)
    cells = to_dev(ram.cells)
    ctx.ram_write(to_dev(ram.addr_trgsw), v, to_dev(ram.new_cell), cells, form=form)
    ctx.sync()
    got = from_dev(cells)
    want = orc.ram_write(p, ram.addr_trgsw, v, ram.new_cell, ram.cells)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("form", FORMS)
def test_ram_write_256_cells(torch_cuda, form):
    p = ti.STD
    ram = ti.ram_write()
    ctx, k = gpu_context(p, ti.SEED_CMUX)
    cells = to_dev(ram.cells)
    ctx.ram_write(to_dev(ram.addr_trgsw), 8, to_dev(ram.new_cell), cells, form=form)
    ctx.sync()
    got = from_dev(cells)
    for c in range(256):
        want = ram.new_bits if c == ram.addr else ram.cell_bits[c]
        assert np.array_equal(orc.trlwe_decrypt(k.s1, got[c])[:32], want[:32]), c
    want = orc.ram_write(p, ram.addr_trgsw, 8, ram.new_cell, ram.cells)
    assert np.array_equal(got, want)
