"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(truth tables, algebraic identities), bounds over all 2^32 inputs, library
routines (numpy convolution), brute force on tiny inputs, and the counts and
sizes printed in the paper's tables (fixtures under tests/golden/).
"""
import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import read_golden

MU = 1 << 29
M32 = 0xFFFFFFFF


def s32(x):
    return np.asarray(x, np.uint32).astype(np.int64) - ((np.asarray(x, np.uint32) >> 31).astype(np.int64) << 32)


def np_negacyclic(a_int, b_u32):
    """a * b mod (X^N + 1, 2^32) with numpy's linear convolution (independent route)."""
    a = np.asarray(a_int, np.int64)
    b = np.asarray(b_u32, np.uint32).astype(np.int64)
    lo = np.convolve(a, b & 0xFFFF)
    hi = np.convolve(a, b >> 16)
    full = (lo.astype(np.uint64) + (hi.astype(np.uint64) << np.uint64(16))) & np.uint64(M32)
    N = a.size
    out = full[:N].copy()
    out[: N - 1] = (out[: N - 1] - full[N:]) & np.uint64(M32)
    return out.astype(np.uint32)


def run_exhaustive(fn, *args):
    """Run a C checker over [0, 2^32) split across threads; returns violations."""
    threads = max(1, min(16, os.cpu_count() or 1))
    step = (1 << 32) // (threads * 8)
    ranges = [(lo, min(1 << 32, lo + step)) for lo in range(0, 1 << 32, step)]
    with ThreadPoolExecutor(threads) as ex:
        return sum(ex.map(lambda r: fn(*args, r[0], r[1]), ranges))


# ---- polynomial arithmetic ---------------------------------------------------------

@pytest.mark.parametrize("N", [2, 4, 16, 256, 1024])
def test_poly_mul_matches_numpy_convolution(N):
    rng = np.random.default_rng(N)
    for a in (rng.integers(-32, 32, N), rng.integers(-(2**31), 2**31, N)):
        b = rng.integers(0, 2**32, N, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(orc.poly_mul(a, b), np_negacyclic(a, b))


def test_poly_mul_brute_force_integers():
    # Z[X] product then reduction by X^N = -1, exact Python integers
    rng = np.random.default_rng(1)
    for N in (1, 2, 3, 5, 8):
        a = [int(x) for x in rng.integers(-100, 100, N)]
        b = [int(x) for x in rng.integers(0, 2**32, N, dtype=np.uint64)]
        prod = [0] * (2 * N)
        for i in range(N):
            for j in range(N):
                prod[i + j] += a[i] * b[j]
        red = [(prod[k] - prod[k + N]) % 2**32 for k in range(N)]
        assert orc.poly_mul(np.array(a), np.array(b, np.uint32)).tolist() == red


@pytest.mark.parametrize("N", [8, 256, 1024])
def test_rotation_identities(N):
    rng = np.random.default_rng(N + 7)
    p = rng.integers(0, 2**32, N, dtype=np.uint64).astype(np.uint32)
    neg = (np.uint32(0) - p).astype(np.uint32)
    assert np.array_equal(orc.rotate(p, 0), p)
    assert np.array_equal(orc.rotate(p, N), neg)                 # X^N = -1
    assert np.array_equal(orc.rotate(orc.rotate(p, N), N), p)    # X^{2N} = 1
    for _ in range(20):
        a, b = (int(x) for x in rng.integers(0, 2 * N, 2))
        assert np.array_equal(orc.rotate(orc.rotate(p, a), b), orc.rotate(p, (a + b) % (2 * N)))
    for k in (1, 3, N - 1, N + 1, 2 * N - 1):
        mono = np.zeros(N, np.int64)
        mono[k % N] = 1 if k < N else -1
        assert np.array_equal(orc.rotate(p, k), np_negacyclic(mono, p))


# ---- rounding steps, exhaustive over all 2^32 Torus32 values ------------------------

def test_decompose_exhaustive(pins_lib):
    fp = orc.fn_address("orc_decompose")
    assert run_exhaustive(pins_lib.chk_decompose, fp, 3, 6) == 0


def test_ks_digits_exhaustive(pins_lib):
    fp = orc.fn_address("orc_ks_digits")
    assert run_exhaustive(pins_lib.chk_ks_digits, fp, 8, 2) == 0
    assert run_exhaustive(pins_lib.chk_ks_digits, fp, 5, 2) == 0


@pytest.mark.parametrize("N", [256, 1024])
def test_modswitch_exhaustive(pins_lib, N):
    assert run_exhaustive(pins_lib.chk_modswitch, orc.fn_address("orc_modswitch"), N) == 0


def test_decompose_special_values():
    # zero decomposes to zero digits (so a zero rotation difference contributes nothing)
    assert orc.decompose(3, 6, 0).tolist() == [0, 0, 0]
    assert orc.decompose(3, 6, 1 << 26).tolist() == [1, 0, 0]          # 1/Bg
    assert orc.decompose(3, 6, (-(1 << 26)) & M32).tolist() == [-1, 0, 0]
    assert orc.decompose(3, 6, 1 << 20).tolist() == [0, 1, 0]          # 1/Bg^2
    assert orc.decompose(3, 6, 1 << 31).tolist() == [-32, 0, 0]        # -1/2
    assert orc.decompose(3, 6, 1 << 13).tolist() == [0, 0, 1]          # tie rounds up
    assert orc.decompose(3, 6, (1 << 13) - 1).tolist() == [0, 0, 0]


def brute_decompose(t, l, Bgbit):
    """Balanced base-Bg digits by repeated division (independent of the oracle)."""
    shift = 32 - l * Bgbit
    r = ((t + (1 << (shift - 1))) >> shift) % (1 << (l * Bgbit))   # round to l*Bgbit bits
    Bg = 1 << Bgbit
    digits = []
    carry = 0
    for _ in range(l):                       # least significant digit first
        d = (r & (Bg - 1)) + carry
        r >>= Bgbit
        if d >= Bg // 2:
            d -= Bg
            carry = 1
        else:
            carry = 0
        digits.append(d)
    return digits[::-1]                      # d_1 (weight 1/Bg) first


def test_decompose_matches_balanced_base_conversion():
    rng = np.random.default_rng(5)
    for t in rng.integers(0, 2**32, 20000, dtype=np.uint64):
        assert orc.decompose(3, 6, int(t)).tolist() == brute_decompose(int(t), 3, 6)


# ---- external product / CMUX -------------------------------------------------------

def gadget_trgsw(p, m):
    """Noiseless TRGSW of m with zero masks: m/Bg^j at coefficient 0 of row j (a) and
    row l+j (b)."""
    C = np.zeros((2 * p.l, 2, p.N), np.uint32)
    for j in range(p.l):
        C[j, 0, 0] = (m << (32 - (j + 1) * p.Bgbit)) & M32
        C[p.l + j, 1, 0] = (m << (32 - (j + 1) * p.Bgbit)) & M32
    return C


def test_external_product_with_gadget_recomposes():
    p = ti.TOY
    rng = np.random.default_rng(2)
    d = rng.integers(0, 2**32, (2, p.N), dtype=np.uint64).astype(np.uint32)
    out1 = orc.external_product(p, gadget_trgsw(p, 1), d)
    err = s32((d.astype(np.int64) - out1.astype(np.int64)) & M32)
    half = 1 << (32 - p.l * p.Bgbit - 1)
    assert err.min() >= -half and err.max() < half
    assert not orc.external_product(p, gadget_trgsw(p, 0), d).any()


def brute_external_product(p, C, d):
    """Python-integer external product for tiny N (independent route)."""
    N, l = p.N, p.l
    out = [[0] * N for _ in range(2)]
    for c in range(2):
        digs = [brute_decompose(int(x), l, p.Bgbit) for x in d[c]]
        for j in range(l):
            row = C[c * l + j]
            poly = [dg[j] for dg in digs]
            for col in range(2):
                for i in range(N):
                    for k in range(N):
                        s = 1 if i + k < N else -1
                        out[col][(i + k) % N] += s * poly[i] * int(row[col][k])
    return np.array([[x % 2**32 for x in r] for r in out], np.uint32)


def test_external_product_brute_force_tiny():
    p = dataclasses.replace(ti.TOY, N=8)
    rng = np.random.default_rng(3)
    for _ in range(5):
        C = rng.integers(0, 2**32, (2 * p.l, 2, p.N), dtype=np.uint64).astype(np.uint32)
        d = rng.integers(0, 2**32, (2, p.N), dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(orc.external_product(p, C, d), brute_external_product(p, C, d))


def test_cmux_selects_with_real_keys():
    p = ti.TOY
    k = ti.keys(p, ti.SEED_TOY)
    rng = np.random.default_rng(4)
    m1 = rng.integers(0, 2, (1, p.N)).astype(np.uint8)
    m0 = rng.integers(0, 2, (1, p.N)).astype(np.uint8)
    d1 = ti.encrypt_trlwe_bits(p, 99, 1, k.s1, m1)[0]
    d0 = ti.encrypt_trlwe_bits(p, 99, 2, k.s1, m0)[0]
    for bit in (0, 1):
        C = ti.encrypt_trgsw_bits(p, 99, 3 + bit, k.s1, [bit])[0]
        got = orc.trlwe_decrypt(k.s1, orc.cmux(p, C, d1, d0))
        assert np.array_equal(got, (m1 if bit else m0)[0])


# ---- BlindRotate ---------------------------------------------------------------------

def test_blind_rotate_every_phase_tiny():
    """Noiseless BSK, n=4, N=16: the accumulator's phase is X^{-phi} v up to the
    decomposition rounding, for every phi in Z_2N."""
    p = ti.Params(n=4, N=16, l=3, Bgbit=6, ks_t=5, ks_basebit=2, sigma0=0.0, sigma1=0.0)
    s0, s1 = ti.keygen(p, 11)
    s0 = np.array([1, 0, 1, 1], np.uint32)
    bsk = ti.make_bsk(p, 11, s0, s1)
    N2 = 2 * p.N
    bound = p.n * (p.N + 1) * (1 << (32 - p.l * p.Bgbit - 1))
    v = np.full(p.N, MU, np.uint32)
    rng = np.random.default_rng(6)
    for phi in range(N2):
        a = rng.integers(0, N2, p.n)
        b = (phi + int((a * s0).sum())) % N2
        acc = orc.blind_rotate(p, bsk, np.concatenate([a, [b]]).astype(np.uint32))
        expect = np.zeros(p.N, np.int64)
        for j in range(p.N):            # coefficient j of X^{-phi} v
            k = (j + phi) % N2
            expect[j] = MU if k < p.N else -MU
        ph = s32(orc.trlwe_phase(s1, acc))
        assert np.abs(ph - expect).max() <= bound, phi


# ---- SampleExtract and key switching -------------------------------------------------

def test_sample_extract_phase_is_coefficient_zero():
    rng = np.random.default_rng(8)
    for N in (8, 256, 1024):
        s = rng.integers(0, 2, N).astype(np.uint32)
        c = rng.integers(0, 2**32, (2, N), dtype=np.uint64).astype(np.uint32)
        tl = orc.sample_extract(c)
        assert orc.tlwe_phase(s, tl) == int(orc.trlwe_phase(s, c)[0])


def test_keyswitch_rounding_with_noiseless_key():
    """With a zero-mask noiseless KSK the output phase is the input phase up to N
    rounding errors of 2^{31 - t basebit}."""
    p = dataclasses.replace(ti.TOY, n=16)
    rng = np.random.default_rng(9)
    s1 = rng.integers(0, 2, p.N).astype(np.uint32)
    s0 = rng.integers(0, 2, p.n).astype(np.uint32)
    base = 1 << p.ks_basebit
    ksk = np.zeros((p.N, p.ks_t, base, p.n + 1), np.uint32)
    for i in range(p.N):
        for j in range(p.ks_t):
            for v in range(1, base):
                ksk[i, j, v, p.n] = (v * int(s1[i]) << (32 - (j + 1) * p.ks_basebit)) & M32
    bound = p.N * (1 << (31 - p.ks_t * p.ks_basebit))
    for _ in range(10):
        c1 = rng.integers(0, 2**32, p.N + 1, dtype=np.uint64).astype(np.uint32)
        out = orc.keyswitch(p, ksk, c1)
        assert not out[: p.n].any()
        err = s32((orc.tlwe_phase(s0, out) - orc.tlwe_phase(s1, c1)) & M32)
        assert abs(int(err)) <= bound


def test_keyswitch_preserves_message_with_real_keys():
    p = ti.TOY
    k = ti.keys(p, ti.SEED_TOY)
    rng = np.random.default_rng(10)
    msg = rng.integers(0, 2, (8, p.N)).astype(np.uint8)
    trl = ti.encrypt_trlwe_bits(p, 5, 5, k.s1, msg)
    for c, m in zip(trl, msg):
        out = orc.keyswitch(p, k.ksk, orc.sample_extract(c))
        assert orc.tlwe_decrypt(k.s0, out) == m[0]


# ---- homomorphic gates ---------------------------------------------------------------

def golden_truth():
    return {row[0]: [int(x) for x in row[1:]] for row in read_golden("gate_truth_tables.txt")}


def test_gate_combine_trivial_inputs_match_truth_tables():
    n = 8
    truth = golden_truth()
    for t, name in enumerate(ti.GATE_NAMES):
        for q, (a, b) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
            c1 = np.zeros(n + 1, np.uint32)
            c2 = np.zeros(n + 1, np.uint32)
            c1[n] = MU if a else (-MU) & M32
            c2[n] = MU if b else (-MU) & M32
            ph = int(s32(orc.gate_combine(n, t, c1, c2)[n]))
            # a nonzero multiple of 1/8 within [-3/8, 3/8] (margin 1/8 from the sign flip)
            assert ph % MU == 0 and ph != 0 and abs(ph) <= 3 * MU
            assert int(ph >= 0) == truth[name][q], (name, a, b)


def test_gate_truth_tables_toy_params():
    truth = golden_truth()
    for seed in (ti.SEED_TOY, ti.SEED_TOY + 100):
        p = ti.TOY
        k = ti.keys(p, seed)
        bits = np.array([0, 0, 0, 1, 1, 0, 1, 1] * 10, np.uint8)
        inp = ti.encrypt_tlwe0_bits(p, seed, 7, k.s0, bits)
        types = np.repeat(np.arange(10, dtype=np.uint8), 4)
        idx = np.arange(80, dtype=np.int32).reshape(40, 2)
        out = orc.gate_batch(p, k.bsk, k.ksk, inp, types, idx)
        dec = orc.tlwe_decrypt(k.s0, out)
        for t, name in enumerate(ti.GATE_NAMES):
            assert dec[4 * t: 4 * t + 4].tolist() == truth[name], name


def test_gate_truth_tables_tfhe_like_params():
    p = ti.STD
    b = ti.flat_level(16)
    gates = [0, 1, 2, 3]
    out = orc.gate_batch(p, b.keys.bsk, b.keys.ksk, b.inp, b.types, b.idx, gates=gates)
    assert np.array_equal(orc.tlwe_decrypt(b.keys.s0, out), b.expected[gates])


def test_gate_rejects_unknown_type():
    with pytest.raises(ValueError):
        orc.gate_combine(4, 10, np.zeros(5), np.zeros(5))


# ---- HomMUX (reading R13) --------------------------------------------------------------

MUX_CASES = [(c, a, b) for c in (0, 1) for a in (0, 1) for b in (0, 1)]


def test_hommux_truth_table_toy_params():
    """MUX(c, a, b) decrypts to c ? a : b for all eight inputs, twice each, real keys."""
    p = ti.TOY
    k = ti.keys(p, ti.SEED_TOY)
    bits = np.array([x for case in MUX_CASES * 2 for x in case], np.uint8)
    inp = ti.encrypt_tlwe0_bits(p, ti.SEED_TOY, 31, k.s0, bits)
    idx = np.arange(3 * 16, dtype=np.int32).reshape(16, 3)
    out = orc.mux_batch(p, k.bsk, k.ksk, inp, idx)
    want = [a if c else b for c, a, b in MUX_CASES * 2]
    assert orc.tlwe_decrypt(k.s0, out).tolist() == want


def test_hommux_without_ks_coefficient_zero_is_the_mux():
    """HomMUX without SE and IKS: coefficient 0 of the TRLWE has phase +1/8 for a 1 and
    -1/8 for a 0, within the bootstrapping noise (far below 1/16)."""
    p = ti.TOY
    k = ti.keys(p, ti.SEED_TOY)
    bits = np.array([x for case in MUX_CASES for x in case], np.uint8)
    inp = ti.encrypt_tlwe0_bits(p, ti.SEED_TOY, 32, k.s0, bits)
    idx = np.arange(24, dtype=np.int32).reshape(8, 3)
    u = orc.mux_batch(p, k.bsk, k.ksk, inp, idx, noks=True)
    for g, (c, a, b) in enumerate(MUX_CASES):
        ph = int(s32(orc.trlwe_phase(k.s1, u[g])[0]))
        want = MU if (a if c else b) else -MU
        assert abs(ph - want) < MU // 2, (c, a, b, ph)


def test_hommux_tfhe_like_params():
    p = ti.STD
    k = ti.keys(p, ti.SEED_FLAT)
    cases = MUX_CASES[1::2]  # four of the eight cases at the full parameters
    bits = np.array([x for case in cases for x in case], np.uint8)
    inp = ti.encrypt_tlwe0_bits(p, ti.SEED_FLAT, 33, k.s0, bits)
    idx = np.arange(3 * len(cases), dtype=np.int32).reshape(len(cases), 3)
    out = orc.mux_batch(p, k.bsk, k.ksk, inp, idx)
    assert orc.tlwe_decrypt(k.s0, out).tolist() == [a if c else b for c, a, b in cases]


def test_mux_batch_rejects_bad_index():
    p = ti.TOY
    k = ti.keys(p, ti.SEED_TOY)
    inp = np.zeros((3, p.n + 1), np.uint32)
    with pytest.raises(ValueError):
        orc.mux_batch(p, k.bsk, k.ksk, inp, np.array([[0, 1, 3]], np.int32))


# ---- CMUX memory ---------------------------------------------------------------------

def test_cmux_tree_reads_every_address_toy():
    rom = ti.cmux_rom(ti.TOY, ti.SEED_TOY, v=4, R=16, packed=ti.TOY.N)
    p = ti.TOY
    for r in range(16):
        orc.extprod_count_reset()
        out = orc.cmux_tree_read(p, rom.addr_trgsw[r], rom.table, 4)
        assert orc.extprod_count() == (1 << 4) - 1
        assert np.array_equal(orc.trlwe_decrypt(rom.keys.s1, out), rom.table_bits[rom.addrs[r]])


def test_ram_write_changes_exactly_the_addressed_cell_toy():
    p = ti.TOY
    k = ti.keys(p, ti.SEED_TOY)
    v = 3
    rng = np.random.default_rng(12)
    cb = rng.integers(0, 2, (1 << v, p.N)).astype(np.uint8)
    cells = ti.encrypt_trlwe_bits(p, 77, 1, k.s1, cb)
    nb = rng.integers(0, 2, (1, p.N)).astype(np.uint8)
    new = ti.encrypt_trlwe_bits(p, 77, 2, k.s1, nb)[0]
    for addr in range(1 << v):
        abits = ((addr >> np.arange(v)) & 1).astype(np.uint8)
        at = ti.encrypt_trgsw_bits(p, 77, 10 + addr, k.s1, abits)
        orc.extprod_count_reset()
        res = orc.ram_write(p, at, v, new, cells)
        assert orc.extprod_count() == (1 << v) * v
        for c in range(1 << v):
            want = nb[0] if c == addr else cb[c]
            assert np.array_equal(orc.trlwe_decrypt(k.s1, res[c]), want), (addr, c)


@pytest.mark.parametrize("flag_bit,stream", [(0, 1), (1, 2), (1, 3)])
def test_ram_cycle_reads_then_writes_the_addressed_word_toy(flag_bit, stream):
    """RAM cycle (reading R14): the read data is the addressed word before the write;
    afterwards coefficient 0 of every refreshed cell decrypts to the old bit, except the
    addressed word, which holds the write data when the flag is 1."""
    p, v, w = ti.TOY, 3, 3
    rc = ti.ram_cycle(p, ti.SEED_TOY, v=v, w=w, flag_bit=flag_bit, stream=stream)
    rd, new = orc.ram_cycle(p, rc.keys.bsk, rc.keys.ksk, rc.addr_trgsw, v, rc.flag, rc.wdata,
                            rc.cells)
    assert orc.tlwe_decrypt(rc.keys.s0, rd).tolist() == rc.cell_bits[:, rc.addr].tolist()
    want = rc.cell_bits.copy()
    if flag_bit:
        want[:, rc.addr] = rc.wdata_bits
    got = np.array([[orc.trlwe_decrypt(rc.keys.s1, new[b, x])[0] for x in range(1 << v)]
                    for b in range(w)])
    assert np.array_equal(got, want)
    # refreshed cells carry +-1/8 at coefficient 0 within bootstrapping noise
    ph = np.array([[int(s32(orc.trlwe_phase(rc.keys.s1, new[b, x])[0])) for x in range(1 << v)]
                   for b in range(w)])
    assert np.all(np.abs(np.abs(ph) - MU) < MU // 4)


def test_packed_rom_reads_every_address_toy():
    """ROM with vertical and horizontal packing (reading R15): every address of a
    32-word x 32-bit ROM (4 TRLWEs of 8 words at N = 256) reads back its word, both as
    the TRLWE's coefficients 0..31 and as 32 TLWE bits."""
    p = ti.TOY
    rom = ti.packed_rom(p, ti.SEED_TOY, M=32, w=32, R=32, stream=5)
    k = rom.keys
    for r in range(32):
        trlwe, bits = orc.rom_read(p, k.ksk, rom.addr_trgsw[r], rom.table, rom.v, rom.w)
        want = rom.words[rom.addrs[r]]
        assert np.array_equal(orc.trlwe_decrypt(k.s1, trlwe)[:32], want), r
        assert np.array_equal(orc.tlwe_decrypt(k.s0, bits), want), r


def test_packed_rom_cmux_count_matches_paper_table():
    """The paper's ROM (512 B: 128 words of 32 bits in 4 TRLWEs at N = 1024) takes 8
    CMUXes per read (Table "The number of CMUXs in CMUX Memory")."""
    p = ti.STD
    rom = ti.packed_rom(p, ti.SEED_CMUX, M=128, w=32, R=1, stream=6)
    assert rom.table.shape == (4, 2, p.N) and rom.v == 7
    orc.extprod_count_reset()
    trlwe, bits = orc.rom_read(p, rom.keys.ksk, rom.addr_trgsw[0], rom.table, rom.v, rom.w)
    assert orc.extprod_count() == 8
    assert np.array_equal(orc.tlwe_decrypt(rom.keys.s0, bits), rom.words[rom.addrs[0]])


def test_cmux_counts_match_paper_table():
    """Per-bit CMUX counts times w reproduce the paper's Read/Write Unit totals."""
    p = ti.TOY
    rows = {r[0]: (int(r[1]), int(r[2]), int(r[3])) for r in read_golden("cmux_memory_counts.txt")}
    w, v, want = rows["ram_read_unit"]
    rom = ti.cmux_rom(p, ti.SEED_TOY, v=v, R=1, packed=8)
    orc.extprod_count_reset()
    orc.cmux_tree_read(p, rom.addr_trgsw[0], rom.table, v)
    assert w * orc.extprod_count() == want
    w, v, want = rows["ram_write_unit"]
    ram = ti.ram_write(p, ti.SEED_TOY, v=v, packed=8)
    orc.extprod_count_reset()
    orc.ram_write(p, ram.addr_trgsw, v, ram.new_cell, ram.cells)
    assert w * orc.extprod_count() == want


def test_ciphertext_sizes_match_paper_table():
    """TRLWE u32[2][N] with N = 1024 gives the paper's RAM and ROM sizes."""
    for name, count, mb in read_golden("ciphertext_sizes.txt"):
        nbytes = int(count) * 2 * ti.STD.N * 4
        digits = len(mb.split(".")[1])
        assert round(nbytes / 1e6, digits) == float(mb), name
