"""CPU model of the packed fp16 arithmetic of the tensor-core digit jobs (csrc/tc.cu:
`digit_pair`, `kara_terms`, `fold_f16_sums`), checked without a GPU against the integer
definitions.

The digit jobs never convert integers to fp16 through the conversion instructions: the
gadget field r (Bgbit bits) of a value is placed under the fp16 bit pattern 0x6600, which
is the number 1536 + r (exponent 10: unit spacing on [1024, 2048)), and one packed
subtraction of 1536 + Bg/2 leaves the signed digit r - Bg/2.  The Karatsuba combinations
are then packed half additions of digits, exact while every value stays within 2048; the
per-block sums of |digit| are kept in packed halves below 512 and read back through the
same pattern (1536 + x has the bit pattern 0x6600 + x).  numpy's float16 is IEEE binary16
with round-to-nearest-even, the rounding of the kernel's add.rn / sub.rn.f16x2.
"""
import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti


def f16_from_bits(b):
    return np.array(b, dtype=np.uint16).view(np.float16)


def bits_of_f16(x):
    return np.array(x, dtype=np.float16).view(np.uint16)


@pytest.mark.parametrize("bgbit", [1, 2, 3, 4, 5, 6])
def test_field_under_0x6600_minus_offset_is_the_signed_digit(bgbit):
    half = 1 << (bgbit - 1)
    raw = np.arange(1 << bgbit, dtype=np.uint16)
    packed = f16_from_bits(raw | 0x6600)
    assert np.array_equal(packed.astype(np.float64), 1536.0 + raw)
    dsub = f16_from_bits(bits_of_f16(np.float16(1536 + half)))
    digit = (packed - dsub).astype(np.float64)
    assert np.array_equal(digit, raw.astype(np.int64) - half)


def test_digit_pair_matches_gadget_digits_of_the_oracle_convention():
    """For l = 3, Bgbit = 6 the fields at bits 26, 20, 14 of u = x + offset, placed under
    0x6600 less 1536 + Bg/2, give the oracle's digits (the gadget decomposition's reading:
    signed [-Bg/2, Bg/2), round to nearest) for random and edge words, and the digits
    recompose the word within half the last digit's weight."""
    p = ti.STD
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.integers(0, 1 << 32, 4096, dtype=np.uint64),
                         np.array([0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF], dtype=np.uint64)]).astype(np.uint32)
    l, bg = p.l, p.Bgbit
    off = sum((1 << (bg - 1)) << (32 - j * bg) for j in range(1, l + 1)) + (1 << (32 - l * bg - 1))
    u = (xs.astype(np.uint64) + off) & 0xFFFFFFFF
    dsub = f16_from_bits(bits_of_f16(np.float16(1536 + (1 << (bg - 1)))))
    for jd in range(l):
        sh = 32 - (jd + 1) * bg
        raw = ((u >> sh) & ((1 << bg) - 1)).astype(np.uint16)
        got = (f16_from_bits(raw | 0x6600) - dsub).astype(np.int64)
        want = np.array([orc.decompose(l, bg, int(x))[jd] for x in xs[:256]])
        assert np.array_equal(got[:256], want)
    digs = []
    for jd in range(l):
        sh = 32 - (jd + 1) * bg
        digs.append(((u >> sh) & ((1 << bg) - 1)).astype(np.int64) - (1 << (bg - 1)))
    rec = sum(d << (32 - (j + 1) * bg) for j, d in enumerate(digs)) & 0xFFFFFFFF
    err = ((rec - xs.astype(np.int64) + (1 << 31)) & 0xFFFFFFFF) - (1 << 31)
    assert np.abs(err).max() <= 1 << (32 - l * bg - 1)


def kara_tree(v, L):
    """The plan's tree on integer blocks v[b] (same order as the kernel's kara_terms):
    negacyclic split x0, x1 - x0, x0 + x1, then per Toeplitz split x0 + x1, x1, x0."""
    def split(blocks):
        if len(blocks) == 1:
            return [blocks[0]]
        h = len(blocks) // 2
        return (split([blocks[i] + blocks[h + i] for i in range(h)]) + split(blocks[h:]) +
                split(blocks[:h]))
    if L == 0:
        return [v[0]]
    h = len(v) // 2
    return (split(v[:h]) + split([v[h + i] - v[i] for i in range(h)]) +
            split([v[i] + v[h + i] for i in range(h)]))


@pytest.mark.parametrize("L", [1, 2, 3])
def test_packed_tree_is_exact(L):
    """Worst-case digits (all -32 or all 31) and random ones: the tree in float16 equals
    the tree in integers, and no combination leaves |x| <= 32 * 2^L (so <= 256)."""
    nb = 1 << L
    rng = np.random.default_rng(L)
    cases = [np.full((nb, 8), -32), np.full((nb, 8), 31), rng.integers(-32, 32, (nb, 8))]
    for x in cases:
        ints = kara_tree([x[b].astype(np.int64) for b in range(nb)], L)
        halves = kara_tree([x[b].astype(np.float16) for b in range(nb)], L)
        assert len(ints) == 3 ** L
        for a, b in zip(ints, halves):
            assert np.abs(a).max() <= 32 * nb
            assert np.array_equal(a, b.astype(np.int64))


def test_tree_rows_are_the_karatsuba_input_combinations():
    """Level 2: the tree's 9 combinations of blocks (x0..x3) are the ones of the
    negacyclic + Toeplitz Karatsuba split (checked on unit vectors)."""
    want = [[1, 1, 0, 0], [0, 1, 0, 0], [1, 0, 0, 0],
            [-1, -1, 1, 1], [0, -1, 0, 1], [-1, 0, 1, 0],
            [1, 1, 1, 1], [0, 1, 0, 1], [1, 0, 1, 0]]
    for b in range(4):
        e = [np.array([1 if k == b else 0]) for k in range(4)]
        got = [int(t[0]) for t in kara_tree(e, 2)]
        assert got == [row[b] for row in want]


def test_fold_of_packed_abs_sums():
    """Sums of |digit| kept in packed halves: up to 3 digits x 4 positions x 32 per half
    (384 < 512) add exactly, and adding 1536 gives the bit pattern 0x6600 + sum."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        d = rng.integers(-32, 32, (12, 2))
        acc = np.zeros(2, dtype=np.float16)
        for row in d:
            acc = (acc + np.abs(row.astype(np.float16))).astype(np.float16)
        assert np.array_equal(acc.astype(np.int64), np.abs(d).sum(0))
        bits = bits_of_f16((acc + np.float16(1536)).astype(np.float16)).astype(np.int64)
        assert np.array_equal(bits - 0x6600, np.abs(d).sum(0))
    worst = np.float16(0)
    for _ in range(12):
        worst = np.float16(worst + np.float16(32))
    assert int(worst) == 384 and int(bits_of_f16(np.float16(worst + np.float16(1536)))) - 0x6600 == 384
