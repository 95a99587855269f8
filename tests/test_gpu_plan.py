"""GPU level scheduler: a layered circuit evaluated level by level (and replayed from
a captured CUDA graph) matches the oracle gate for gate."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu


def oracle_circuit(p, k, c, inp):
    wires = np.zeros((c.num_inputs + c.num_gates, p.n + 1), np.uint32)
    wires[: c.num_inputs] = inp
    for L in range(int(c.level.max()) + 1):
        gs = np.nonzero(c.level == L)[0]
        out = orc.gate_batch(p, k.bsk, k.ksk, wires, c.types, c.idx, gates=gs)
        wires[c.num_inputs + gs] = out
    return wires[c.num_inputs:]


@pytest.mark.parametrize("form", [-1, 0, 2])
def test_toy_dag_matches_oracle(torch_cuda, form):
    import paper_2010_09410_b300 as tb
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    circs = [ti.layered_dag(ti.SEED_TOY, total=150, levels=8, num_inputs=16, lo=5, hi=40, stream=s)
             for s in (1, 2)]
    ins = [ti.encrypt_tlwe0_bits(p, ti.SEED_TOY, 50 + i, k.s0,
                                 ti.random_bits(ti.SEED_TOY, 60 + i, c.num_inputs))
           for i, c in enumerate(circs)]
    plan = ctx.plan(circs, form)
    assert 1 <= plan.num_levels <= 8
    out = torch_cuda.zeros((sum(c.num_gates for c in circs), p.n + 1), dtype=torch_cuda.int32,
                           device="cuda")
    plan.run(to_dev(np.concatenate(ins)), out)
    ctx.sync()
    got = from_dev(out)
    want = np.concatenate([oracle_circuit(p, k, c, x) for c, x in zip(circs, ins)])
    assert np.array_equal(got, want)
    out2 = torch_cuda.zeros_like(out)
    dev_in = to_dev(np.concatenate(ins))
    plan.run(dev_in, out2, use_graph=True)
    plan.run(dev_in, out2, use_graph=True)
    ctx.sync()
    assert np.array_equal(from_dev(out2), want)
    # a wider batch reallocates the context's workspaces; the plan must notice and
    # record its graph again instead of replaying stale addresses
    G = 5000  # wider than any toy batch of the other tests
    bits = ti.random_bits(ti.SEED_TOY, 70, 2 * G)
    b_in = to_dev(ti.encrypt_tlwe0_bits(p, ti.SEED_TOY, 71, k.s0, bits))
    b_types = to_dev(ti.random_below(ti.SEED_TOY, 72, G, 10).astype(np.uint8))
    b_idx = to_dev(np.arange(2 * G, dtype=np.int32).reshape(G, 2))
    b_out = torch_cuda.zeros((G, p.n + 1), dtype=torch_cuda.int32, device="cuda")
    ctx.gate_batch(b_in, b_types, b_idx, b_out, form=max(form, 0))
    out3 = torch_cuda.zeros_like(out)
    plan.run(dev_in, out3, use_graph=True)
    ctx.sync()
    assert np.array_equal(from_dev(out3), want)


def test_toy_dag_dataflow_matches_oracle(torch_cuda):
    """The dataflow run (each gate started once its inputs exist, two-prime per-gate
    form) gives the oracle's words, twice in a row (the queues and counters are reset
    per run)."""
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    circs = [ti.layered_dag(ti.SEED_TOY, total=150, levels=8, num_inputs=16, lo=5, hi=40, stream=s)
             for s in (1, 2)]
    ins = [ti.encrypt_tlwe0_bits(p, ti.SEED_TOY, 50 + i, k.s0,
                                 ti.random_bits(ti.SEED_TOY, 60 + i, c.num_inputs))
           for i, c in enumerate(circs)]
    plan = ctx.plan(circs)
    want = np.concatenate([oracle_circuit(p, k, c, x) for c, x in zip(circs, ins)])
    dev_in = to_dev(np.concatenate(ins))
    for _ in range(2):
        out = torch_cuda.zeros((sum(c.num_gates for c in circs), p.n + 1), dtype=torch_cuda.int32,
                               device="cuda")
        plan.run_dataflow(dev_in, out)
        ctx.sync()
        assert np.array_equal(from_dev(out), want)


def test_dataflow_chain_and_fan_in(torch_cuda):
    """Degenerate DAGs: a chain of 12 gates (one ready gate at a time, every other block
    waits), a gate reading the same gate twice, and gates reading only primaries."""
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    ni, G = 4, 16
    types = (np.arange(G) % 10).astype(np.uint8)
    idx = np.zeros((G, 2), np.int32)
    idx[0] = (0, 1)
    for g in range(1, 12):
        idx[g] = (ni + g - 1, g % ni)            # chain through the previous gate
    idx[12] = (ni + 11, ni + 11)                 # the same gate twice
    idx[13] = (2, 3)                             # primaries only
    idx[14] = (ni + 13, ni + 12)
    idx[15] = (0, ni + 14)

    class C:
        pass
    c = C()
    c.num_inputs, c.num_gates, c.types, c.idx = ni, G, types, idx
    lv = np.zeros(G, int)
    for g in range(G):
        lv[g] = max([lv[w - ni] + 1 for w in idx[g] if w >= ni] + [0])
    c.level = lv
    x = ti.encrypt_tlwe0_bits(p, ti.SEED_TOY, 80, k.s0, ti.random_bits(ti.SEED_TOY, 81, ni))
    plan = ctx.plan([c])
    out = torch_cuda.zeros((G, p.n + 1), dtype=torch_cuda.int32, device="cuda")
    plan.run_dataflow(to_dev(x), out)
    ctx.sync()
    assert np.array_equal(from_dev(out), oracle_circuit(p, k, c, x))
