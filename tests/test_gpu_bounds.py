"""The debug build (libtfhe_b300_bounds.so, compiled with TFHE_BOUNDS_CHECK): device index
checks on the hot path (tensor-core BlindRotate: digit stores, accumulator loads, stores and
reductions, combination words, bulk-copy sources, line discards; dataflow engine: wire,
consumer and queue indices) record TFHE_EBOUNDS instead of touching memory out of range.
Run in a child process (the binding loads one library per process) over the paths at sizes
with ragged tails, it must report no violation and give the oracle's words."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np
import oracle as orc
import tfhe_inputs as ti
import paper_2010_09410_b300 as tb
from conftest import from_dev, gpu_context, to_dev
import torch
assert tb.LIB_PATH.endswith("libtfhe_b300_bounds.so"), tb.LIB_PATH

def empty(G, w):
    return torch.zeros((G, w), dtype=torch.int32, device="cuda")

# toy gates in every form, word for word
p = ti.TOY
ctx, k = gpu_context(p, ti.SEED_TOY)
b = ti.toy_gates()
want = orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx)
for form in (0, 1, 2):
    out = empty(b.types.size, p.n + 1)
    ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
    ctx.sync()
    assert np.array_equal(from_dev(out), want), form

# tensor-core CMUX mode with a ragged group
rng = np.random.default_rng(1)
B, group = 350, 150
sel = ti.encrypt_trgsw_bits(p, 7, 3, k.s1, rng.integers(0, 2, 3).astype(np.uint8))
d1 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
d0 = rng.integers(0, 2**32, (B, 2, p.N), dtype=np.uint64).astype(np.uint32)
out = to_dev(np.zeros_like(d0))
ctx.cmux_batch(to_dev(sel), group, to_dev(d1), to_dev(d0), out, form=1)
ctx.sync()
got = from_dev(out)
for q in (0, 149, 150, 299, 300, 349):
    assert np.array_equal(got[q], orc.cmux(p, sel[q // group], d1[q], d0[q])), q

# toy DAG: dataflow run equals the level run
circs = [ti.layered_dag(ti.SEED_TOY, total=150, levels=8, num_inputs=16, lo=5, hi=40, stream=1)]
x = ti.encrypt_tlwe0_bits(p, ti.SEED_TOY, 50, k.s0, ti.random_bits(ti.SEED_TOY, 60, circs[0].num_inputs))
plan = ctx.plan(circs)
o1, o2 = empty(150, p.n + 1), empty(150, p.n + 1)
plan.run(to_dev(x), o1)
plan.run_dataflow(to_dev(x), o2)
ctx.sync()
assert torch.equal(o1, o2)

# the TFHE-like parameters: 300 gates (three tiles, a ragged last one) at Karatsuba
# levels 2 and 3, and forced two passes
p = ti.STD
ctx, k = gpu_context(p, ti.SEED_FLAT)
b = ti.flat_level(300)
sample = [0, 127, 128, 255, 256, 299]
want = orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx, gates=sample)
for level, limit in ((2, -1), (3, -1), (2, 0)):
    ctx.set_tc_level(level)
    ctx.set_tc_pass_limit(limit)
    out = empty(300, p.n + 1)
    ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=1)
    ctx.sync()
    got = from_dev(out)
    assert np.array_equal(orc.tlwe_decrypt(k.s0, got), b.expected), level
    assert np.array_equal(got[sample], want), level
ctx.set_tc_level(-1)
ctx.set_tc_pass_limit(-1)
print("bounds ok")
'''


def test_debug_build_reports_no_bounds_violation():
    lib = os.path.join(ROOT, "paper_2010_09410_b300", "libtfhe_b300_bounds.so")
    assert os.path.exists(lib), "the debug build is made by __graft_entry__.build()"
    env = dict(os.environ, TFHE_B300_BOUNDS="1",
               PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "bounds ok" in r.stdout
