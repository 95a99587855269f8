"""GPU parity of bootstrapped gates, BlindRotate and key switching against the CPU
oracle: every output word bit-exact (all arithmetic is mod 2^32)."""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import from_dev, gpu_context, to_dev

pytestmark = pytest.mark.gpu

FORMS = [0, 1, 2, -1]


def empty(torch, *shape):
    return torch.zeros(shape, dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("form", FORMS)
def test_toy_gates_bit_exact(torch_cuda, form):
    b = ti.toy_gates()
    ctx, k = gpu_context(ti.TOY, ti.SEED_TOY)
    out = empty(torch_cuda, b.types.size, ti.TOY.n + 1)
    ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
    ctx.sync()
    got = from_dev(out)
    want = orc.gate_batch(ti.TOY, k.bsk, k.ksk, b.inp, b.types, b.idx)
    assert np.array_equal(got, want)
    assert np.array_equal(orc.tlwe_decrypt(k.s0, got), b.expected)


@pytest.mark.parametrize("form", FORMS)
def test_blind_rotate_stage_toy(torch_cuda, form):
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    rng = np.random.default_rng(1)
    G = 19
    bar = rng.integers(0, 2 * p.N, (G, p.n + 1)).astype(np.uint32)
    bar[3, :] = 0                  # all rotations zero
    bar[4, :-1] = 0                # only b~ nonzero
    bar[5, -1] = 2 * p.N - 1
    acc = empty(torch_cuda, G, 2, p.N)
    ctx.blind_rotate(to_dev(bar), acc, form=form)
    ctx.sync()
    got = from_dev(acc)
    for g in range(G):
        assert np.array_equal(got[g], orc.blind_rotate(p, k.bsk, bar[g])), g


def test_extract_keyswitch_stage_toy(torch_cuda):
    p = ti.TOY
    ctx, k = gpu_context(p, ti.SEED_TOY)
    rng = np.random.default_rng(2)
    G = 21                          # not a multiple of the 8-gate key-switch tile
    acc = rng.integers(0, 2**32, (G, 2, p.N), dtype=np.uint64).astype(np.uint32)
    out = empty(torch_cuda, G, p.n + 1)
    ctx.extract_keyswitch(to_dev(acc), out)
    ctx.sync()
    got = from_dev(out)
    for g in range(G):
        want = orc.keyswitch(p, k.ksk, orc.sample_extract(acc[g]))
        assert np.array_equal(got[g], want), g


@pytest.mark.parametrize("form", FORMS)
def test_tfhe_like_gates_ragged_batch(torch_cuda, form):
    """37 gates at n=630, N=1024: spans several key-switch tiles plus a ragged tail;
    every output word compared with the oracle."""
    b = ti.flat_level(37)
    ctx, k = gpu_context(ti.STD, ti.SEED_FLAT)
    out = empty(torch_cuda, 37, ti.STD.n + 1)
    ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
    ctx.sync()
    got = from_dev(out)
    want = orc.gate_batch(ti.STD, k.bsk, k.ksk, b.inp, b.types, b.idx)
    assert np.array_equal(got, want)
    assert np.array_equal(orc.tlwe_decrypt(k.s0, got), b.expected)


_FLAT_SAMPLE = {}


def flat_level_sample(k, b):
    """256 seeded gates of the 4096-gate level: the first and last gate of every 128-gate
    tile (64) plus 192 drawn without repetition from the rest; with the oracle's words for
    them (computed once for every form)."""
    if "want" not in _FLAT_SAMPLE:
        G = b.types.size
        edges = sorted({g for t in range(0, G, 128) for g in (t, min(t + 127, G - 1))})
        rest = np.setdiff1d(np.arange(G), edges)
        extra = np.random.default_rng(3).choice(rest, 256 - len(edges), replace=False)
        sample = sorted(set(edges) | set(int(g) for g in extra))
        assert len(sample) == 256
        _FLAT_SAMPLE["gates"] = sample
        _FLAT_SAMPLE["want"] = orc.gate_batch(ti.STD, k.bsk, k.ksk, b.inp, b.types, b.idx,
                                              gates=sample)
    return _FLAT_SAMPLE["gates"], _FLAT_SAMPLE["want"]


@pytest.mark.parametrize("form", FORMS)
def test_flat_level_4096_sampled(torch_cuda, form):
    """The full 4096-gate level in the benchmark's launch configuration: all outputs
    decrypt to the plaintext gates, and 256 seeded gates (among them the first and last
    gate of every 128-gate tile) match the oracle word for word."""
    b = ti.flat_level(4096)
    ctx, k = gpu_context(ti.STD, ti.SEED_FLAT)
    out = empty(torch_cuda, 4096, ti.STD.n + 1)
    ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
    ctx.sync()
    got = from_dev(out)
    assert np.array_equal(orc.tlwe_decrypt(k.s0, got), b.expected)
    sample, want = flat_level_sample(k, b)
    bad = [g for g, w in zip(sample, want) if not np.array_equal(got[g], w)]
    assert not bad, bad[:10]


@pytest.mark.parametrize("G", [149, 301])
def test_two_prime_form_wider_than_the_sms(torch_cuda, G):
    """Levels wider than the SM count run the two-prime form as two 512-thread blocks per
    SM, at odd widths too.  Every word equals the NTT form's over 2^64 - 2^32 + 1 (an
    independent product), all outputs decrypt to the plaintext gates, and the first, a
    middle and the last two gates match the oracle word for word."""
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_FLAT)
    b = ti.flat_level(G)
    outs = {}
    for form in (0, 2):
        out = empty(torch_cuda, G, p.n + 1)
        ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
        ctx.sync()
        outs[form] = from_dev(out)
    assert np.array_equal(outs[2], outs[0])
    assert np.array_equal(orc.tlwe_decrypt(k.s0, outs[2]), b.expected)
    sample = [0, G // 2, G - 2, G - 1]
    want = orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx, gates=sample)
    assert np.array_equal(outs[2][sample], want)


def test_zero_gates_is_noop(torch_cuda):
    ctx, k = gpu_context(ti.TOY, ti.SEED_TOY)
    t = empty(torch_cuda, 0)
    ctx.gate_batch(empty(torch_cuda, 1, ti.TOY.n + 1), t.to(torch_cuda.uint8), t, t)
    ctx.sync()


@pytest.mark.parametrize("form", [0, 1])
def test_bad_type_and_index_reported_on_device(torch_cuda, form):
    """A bad gate type and an out-of-range input index are caught on the device: those
    gates give all-zero outputs, TFHE_EINVAL comes back at the next sync, and every other
    gate is still bit-exact (form 1: the tensor-core BlindRotate forms the combinations
    itself)."""
    b = ti.toy_gates()
    ctx, k = gpu_context(ti.TOY, ti.SEED_TOY)
    types = b.types.copy()
    idx = b.idx.copy()
    types[2] = 10
    idx[5, 1] = 1000
    out = empty(torch_cuda, types.size, ti.TOY.n + 1)
    ctx.gate_batch(to_dev(b.inp), to_dev(types), to_dev(idx), out, form=form)
    import paper_2010_09410_b300 as tb
    with pytest.raises(tb.TfheError) as e:
        ctx.sync()
    assert e.value.code == -1
    got = from_dev(out)
    assert not got[2].any() and not got[5].any()
    good = [g for g in range(types.size) if g not in (2, 5)]
    want = orc.gate_batch(ti.TOY, k.bsk, k.ksk, b.inp, b.types, b.idx, gates=good)
    assert np.array_equal(got[good], want)
    ctx.sync()                          # the error word was cleared


def test_host_buffer_entry_point_matches_device(torch_cuda):
    b = ti.toy_gates()
    ctx, k = gpu_context(ti.TOY, ti.SEED_TOY)
    out = np.zeros((b.types.size, ti.TOY.n + 1), np.uint32)
    ctx.gate_batch_host(b.inp, b.types, np.ascontiguousarray(b.idx), out)
    want = orc.gate_batch(ti.TOY, k.bsk, k.ksk, b.inp, b.types, b.idx)
    assert np.array_equal(out, want)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("params,seed,levels,G", [
    (ti.TOY, ti.SEED_TOY, (0, 1), 40),
    (ti.STD, ti.SEED_FLAT, (0, 1, 2, 3), 37),
])
def test_tc_karatsuba_levels_bit_exact(torch_cuda, params, seed, levels, G, variant):
    """Every Karatsuba level of the tensor-core form, on one SM per tile and on SM pairs,
    gives the oracle's words."""
    ctx, k = gpu_context(params, seed)
    b = ti.toy_gates() if params is ti.TOY else ti.flat_level(G)
    want = orc.gate_batch(params, k.bsk, k.ksk, b.inp, b.types, b.idx)
    try:
        ctx.set_tc_variant(variant)
        assert ctx.tc_variant() == variant
        for L in levels:
            ctx.set_tc_level(L)
            out = empty(torch_cuda, b.types.size, params.n + 1)
            ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=1)
            ctx.sync()
            assert np.array_equal(from_dev(out), want), L
    finally:
        ctx.set_tc_level(-1)
        ctx.set_tc_variant(-1)


@pytest.mark.parametrize("limit", [0, 60000])
@pytest.mark.parametrize("params,seed,G,level", [(ti.TOY, ti.SEED_TOY, 40, -1),
                                                 (ti.STD, ti.SEED_FLAT, 300, -1),
                                                 (ti.STD, ti.SEED_FLAT, 300, 3)])
def test_tc_one_and_two_pass_accumulation(torch_cuda, params, seed, G, level, limit):
    """Steps accumulated in two TMEM passes (forced everywhere with limit 0, mixed with
    one-pass steps at 60000) give the same words as the default; sampled gates match the
    oracle.  Level 3 bounds the one-pass sum through per-block digit sums."""
    ctx, k = gpu_context(params, seed)
    b = ti.toy_gates() if params is ti.TOY else ti.flat_level(G)
    outs = []
    if level >= 0:
        ctx.set_tc_level(level)
    try:
        for lim in (-1, limit):
            ctx.set_tc_pass_limit(lim)
            out = empty(torch_cuda, b.types.size, params.n + 1)
            ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=1)
            ctx.sync()
            outs.append(from_dev(out))
    finally:
        ctx.set_tc_pass_limit(-1)
        ctx.set_tc_level(-1)
    assert np.array_equal(outs[0], outs[1])
    samples = [0, b.types.size // 2, b.types.size - 1]
    want = orc.gate_batch(params, k.bsk, k.ksk, b.inp, b.types, b.idx, gates=samples)
    assert np.array_equal(outs[1][samples], want)


def test_tc_pass_limit_rejects_inexact_values(torch_cuda):
    import paper_2010_09410_b300 as tb
    ctx, _ = gpu_context(ti.STD, ti.SEED_FLAT)
    with pytest.raises(tb.TfheError):
        ctx.set_tc_pass_limit((1 << 17) + 1)


@pytest.mark.parametrize("G", [300, 129, 1000])
def test_tc_variants_agree_on_every_word(torch_cuda, G):
    """One-SM and SM-pair BlindRotate give the same words for all gates, including tile
    counts that leave the last pair half empty (3 and 2 tiles of 128 gates, 8 tiles with
    a ragged last one); sampled gates, first and last of every tile, match the oracle."""
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_FLAT)
    b = ti.flat_level(G)
    outs = {}
    try:
        for v in (0, 1):
            ctx.set_tc_variant(v)
            out = empty(torch_cuda, G, p.n + 1)
            ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=1)
            ctx.sync()
            outs[v] = from_dev(out)
    finally:
        ctx.set_tc_variant(-1)
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(orc.tlwe_decrypt(k.s0, outs[1]), b.expected)
    samples = sorted({g for t in range(0, G, 128) for g in (t, min(t + 127, G - 1))})
    want = orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx, gates=samples)
    assert np.array_equal(outs[1][samples], want)


def test_tc_uneven_tile_chunks(torch_cuda):
    """4,224 gates = 33 tiles: the tensor-core launch runs its tiles in two chunks of 17
    and 16 (all steps of one chunk before the next).  Every output decrypts to its
    plaintext gate, the first and last gate of every tile match the oracle word for word,
    and the words equal the two-prime per-gate form's."""
    p = ti.STD
    ctx, k = gpu_context(p, ti.SEED_FLAT)
    G = 4224
    b = ti.flat_level(G)
    outs = {}
    for form in (1, 2):
        out = empty(torch_cuda, G, p.n + 1)
        ctx.gate_batch(to_dev(b.inp), to_dev(b.types), to_dev(b.idx), out, form=form)
        ctx.sync()
        outs[form] = from_dev(out)
    assert np.array_equal(orc.tlwe_decrypt(k.s0, outs[1]), b.expected)
    assert np.array_equal(outs[1], outs[2])
    samples = sorted({g for t in range(0, G, 128) for g in (t, min(t + 127, G - 1))})
    want = orc.gate_batch(p, k.bsk, k.ksk, b.inp, b.types, b.idx, gates=samples)
    assert np.array_equal(outs[1][samples], want)
