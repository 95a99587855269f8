"""GPU RAM cycle (Section 8.2: read unit, control unit, write unit with refresh) against
the oracle: read data and every refreshed cell bit-exact."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu


def run_cycle(torch, ctx, p, rc, v, form):
    cells = to_dev(rc.cells)
    rdata = torch.zeros((rc.w, p.n + 1), dtype=torch.int32, device="cuda")
    ctx.ram_cycle(to_dev(rc.addr_trgsw), v, to_dev(rc.flag), to_dev(rc.wdata), cells, rdata,
                  form=form)
    ctx.sync()
    return from_dev(rdata), from_dev(cells)


@pytest.mark.parametrize("form", [0, 1, 2, -1])
@pytest.mark.parametrize("flag_bit,stream", [(0, 11), (1, 12)])
def test_ram_cycle_toy_bit_exact(torch_cuda, form, flag_bit, stream):
    p, v, w = ti.TOY, 3, 3
    ctx, k = gpu_context(p, ti.SEED_TOY)
    rc = ti.ram_cycle(p, ti.SEED_TOY, v=v, w=w, flag_bit=flag_bit, stream=stream)
    rd, cells = run_cycle(torch_cuda, ctx, p, rc, v, form)
    want_rd, want_cells = orc.ram_cycle(p, k.bsk, k.ksk, rc.addr_trgsw, v, rc.flag, rc.wdata,
                                        rc.cells)
    assert np.array_equal(rd, want_rd)
    assert np.array_equal(cells, want_cells)
    assert orc.tlwe_decrypt(k.s0, rd).tolist() == rc.cell_bits[:, rc.addr].tolist()


def test_ram_cycle_tfhe_like_params(torch_cuda):
    p, v, w = ti.STD, 2, 2
    ctx, k = gpu_context(p, ti.SEED_CMUX)
    rc = ti.ram_cycle(p, ti.SEED_CMUX, v=v, w=w, flag_bit=1, stream=13)
    rd, cells = run_cycle(torch_cuda, ctx, p, rc, v, 1)
    want_rd, want_cells = orc.ram_cycle(p, k.bsk, k.ksk, rc.addr_trgsw, v, rc.flag, rc.wdata,
                                        rc.cells)
    assert np.array_equal(rd, want_rd)
    assert np.array_equal(cells, want_cells)
    want = rc.cell_bits.copy()
    want[:, rc.addr] = rc.wdata_bits
    got = np.array([[orc.trlwe_decrypt(k.s1, cells[b, x])[0] for x in range(1 << v)]
                    for b in range(w)])
    assert np.array_equal(got, want)
