"""Whole circuits at the paper's parameters through the level scheduler (circuit
evaluation by levels, Section 6.2; gates of one level are independent, so a level is
one batch).

Two workloads: a layered DAG of 20,000 gates over 60 levels with 256 primary inputs
(every gate input drawn from the previous three levels or the primaries), and 16
independent layered circuits of 2,000-40,000 gates and 20-120 levels interleaved level
by level.  The oracle cannot evaluate 10^4-10^5 bootstrapped gates in a test, so each
run is checked two ways that hold at any size:

* every gate output decrypts to the plaintext circuit evaluated on the plaintext bits;
* sampled gates, spread over the levels (wide levels run in the tensor-core form, narrow
  ones in the NTT form), are recomputed one by one by the oracle from the GPU's own
  input wires and must match bit for bit.
"""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu

TRUTH = np.array([[[ti.plain_gate(t, a, b) for b in (0, 1)] for a in (0, 1)]
                  for t in range(10)], np.uint8)


def plain_eval(c, in_bits):
    """Plaintext value of every gate output (gates are stored in level order)."""
    wires = np.concatenate([in_bits.astype(np.uint8), np.zeros(c.num_gates, np.uint8)])
    for L in range(int(c.level.max()) + 1):
        gs = np.nonzero(c.level == L)[0]
        a = wires[c.idx[gs, 0]]
        b = wires[c.idx[gs, 1]]
        wires[c.num_inputs + gs] = TRUTH[c.types[gs], a, b]
    return wires[c.num_inputs:]


def longest_path_levels(c):
    """Level of every gate as the scheduler defines it: the longest path from the
    primary inputs (a gate fed only by primaries is at level 0)."""
    lv = np.full(c.num_inputs + c.num_gates, -1, np.int64)
    for g in range(c.num_gates):  # inputs always precede the gate
        lv[c.num_inputs + g] = max(lv[c.idx[g, 0]], lv[c.idx[g, 1]]) + 1
    return lv[c.num_inputs:]


def sample_gates(lv, per_level_step, seed_stream):
    """Two gates from every `per_level_step`-th scheduler level, chosen reproducibly."""
    rng = ti.random_u64(ti.SEED_DAG, seed_stream, 2 * (int(lv.max()) + 1))
    out = []
    for L in range(0, int(lv.max()) + 1, per_level_step):
        gs = np.nonzero(lv == L)[0]
        for j in range(2):
            out.append(int(gs[int(rng[2 * L + j] % np.uint64(gs.size))]))
    return sorted(set(out))


def check_circuit(p, k, c, in_ct, in_bits, got, samples):
    dec = orc.tlwe_decrypt(k.s0, got)
    want_bits = plain_eval(c, in_bits)
    assert np.array_equal(dec, want_bits), np.nonzero(dec != want_bits)[0][:10]
    wires = np.concatenate([in_ct, got])
    ref = orc.gate_batch(p, k.bsk, k.ksk, wires, c.types, c.idx, gates=samples)
    assert np.array_equal(ref, got[samples]), samples


def test_dag_20000_gates_60_levels(torch_cuda):
    torch = torch_cuda
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_FLAT)
    c = ti.layered_dag(ti.SEED_DAG)
    assert c.num_gates == 20000 and int(c.level.max()) == 59
    bits = ti.random_bits(ti.SEED_DAG, 900, c.num_inputs)
    in_ct = ti.encrypt_tlwe0_bits(p, ti.SEED_DAG, 901, k.s0, bits)
    plan = ctx.plan([c])
    lv = longest_path_levels(c)
    assert plan.num_levels == int(lv.max()) + 1
    out = torch.zeros((c.num_gates, p.n + 1), dtype=torch.int32, device="cuda")
    dev_in = to_dev(in_ct)
    plan.run(dev_in, out)
    ctx.sync()
    got = from_dev(out)
    widths = np.bincount(lv)
    samples = sample_gates(lv, 4, 902)
    # both forms are exercised: some sampled levels are narrower than the tensor-core
    # threshold, some wider
    assert widths[lv[samples]].min() < 128 <= widths[lv[samples]].max()
    check_circuit(p, k, c, in_ct, bits, got, samples)
    # a replay of the captured graph gives the same words
    out2 = torch.zeros_like(out)
    plan.run(dev_in, out2, use_graph=True)
    ctx.sync()
    assert torch.equal(out, out2)
    # the dataflow run gives the same words (all gates in the two-prime per-gate form)
    out3 = torch.zeros_like(out)
    plan.run_dataflow(dev_in, out3)
    ctx.sync()
    assert torch.equal(out, out3)


def test_16_mixed_circuits_interleaved(torch_cuda):
    torch = torch_cuda
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_FLAT)
    circs = ti.mixed_circuits()
    assert len(circs) == 16
    bits = [ti.random_bits(ti.SEED_MIXED, 910 + i, c.num_inputs) for i, c in enumerate(circs)]
    cts = [ti.encrypt_tlwe0_bits(p, ti.SEED_MIXED, 930 + i, k.s0, b) for i, b in enumerate(bits)]
    plan = ctx.plan(circs)
    lvs = [longest_path_levels(c) for c in circs]
    last = [int(lv.max()) for lv in lvs]
    assert plan.num_levels == max(last) + 1
    assert plan.circuit_last_level == last
    total = sum(c.num_gates for c in circs)
    out = torch.zeros((total, p.n + 1), dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(plan.num_levels)]
    start = torch.cuda.Event(enable_timing=True)
    dev_in = to_dev(np.concatenate(cts))
    start.record()
    plan.run(dev_in, out, level_events=ev)
    ctx.sync()
    torch.cuda.synchronize()
    # per-circuit completion: a circuit is done when its last level is
    done_ms = [start.elapsed_time(ev[L]) for L in plan.circuit_last_level]
    assert all(t > 0 for t in done_ms)
    assert max(done_ms) == pytest.approx(start.elapsed_time(ev[-1]))
    got = from_dev(out)
    off = 0
    for i, c in enumerate(circs):
        g = got[off: off + c.num_gates]
        off += c.num_gates
        samples = sample_gates(lvs[i], 40, 940 + i)[:3]
        check_circuit(p, k, c, cts[i], bits[i], g, samples)
    # the dataflow run gives the same words for all 16 circuits at once
    out2 = torch.zeros_like(out)
    plan.run_dataflow(dev_in, out2)
    ctx.sync()
    assert torch.equal(out, out2)


def test_autotuned_plan_matches_fixed_forms(torch_cuda):
    """The autotuner's table covers the width ladder with valid choices, and a plan that
    follows it (per-level form and Karatsuba level) gives the same words as plans fixed
    to each form."""
    torch = torch_cuda
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_FLAT)
    table = ctx.autotune(512)
    assert [w for w, _, _, _ in table] == [64, 128, 256, 512]
    for w, form, level, ms in table:
        assert form in (0, 1, 2) and ms > 0
        assert (form in (0, 2) and level == -1) or (form == 1 and level in (0, 1, 2))
    c = ti.layered_dag(ti.SEED_DAG, total=2400, levels=6, num_inputs=256, lo=50, hi=800, stream=7)
    bits = ti.random_bits(ti.SEED_DAG, 990, c.num_inputs)
    dev_in = to_dev(ti.encrypt_tlwe0_bits(p, ti.SEED_DAG, 991, k.s0, bits))
    outs = []
    for form in (-1, 0, 1, 2):
        plan = ctx.plan([c], form)
        out = torch.zeros((c.num_gates, p.n + 1), dtype=torch.int32, device="cuda")
        plan.run(dev_in, out)
        ctx.sync()
        outs.append(from_dev(out))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    assert np.array_equal(orc.tlwe_decrypt(k.s0, outs[0]), plain_eval(c, bits))
