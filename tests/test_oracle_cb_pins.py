"""Pins of the oracle's circuit bootstrapping (reading R16) and its Torus64 primitives.

Each test checks the oracle against something other than itself: Python-integer brute
force and limb-wise numpy convolutions for the 64-bit negacyclic product, algebraic
identities of the rotation, balanced base conversion for the gadget digits, analytic
rounding bounds for BlindRotate and the private key switch with noiseless keys,
decryption of every circuit-bootstrapped TRGSW row, the CMUX and CMUX tree driven by
circuit-bootstrapped addresses, and the paper's printed bootstrapping-key size.
"""
import dataclasses

import numpy as np
import pytest

import oracle as orc
import tfhe_inputs as ti
from conftest import read_golden

M32 = 0xFFFFFFFF
M64 = (1 << 64) - 1


def s64(x: int) -> int:
    x &= M64
    return x - (1 << 64) if x >> 63 else x


def s32(x: int) -> int:
    x &= M32
    return x - (1 << 32) if x >> 31 else x


def rand_u64(rng, shape):
    return rng.integers(0, 2**64, shape, dtype=np.uint64)


def brute_negacyclic64(a, b):
    N = len(a)
    prod = [0] * (2 * N)
    for i in range(N):
        for j in range(N):
            prod[i + j] += int(a[i]) * int(b[j])
    return [(prod[k] - prod[k + N]) % 2**64 for k in range(N)]


def limb_negacyclic64(a, b):
    """a * b mod (X^N + 1, 2^64) from four int64 convolutions of 16-bit limbs of b."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.uint64)
    N = a.size
    full = np.zeros(2 * N - 1, np.uint64)
    for k in range(4):
        limb = ((b >> np.uint64(16 * k)) & np.uint64(0xFFFF)).astype(np.int64)
        full += np.convolve(a, limb).astype(np.uint64) << np.uint64(16 * k)  # wraps mod 2^64
    out = full[:N].copy()
    out[: N - 1] -= full[N:]
    return out


# ---- Torus64 polynomial arithmetic -------------------------------------------------

def test_poly_mul64_brute_force_integers():
    rng = np.random.default_rng(21)
    for N in (1, 2, 3, 5, 8, 16):
        a = rng.integers(-256, 256, N)
        b = rand_u64(rng, N)
        assert orc.poly_mul64(a, b).tolist() == brute_negacyclic64(a, b)


@pytest.mark.parametrize("N", [16, 512, 2048])
def test_poly_mul64_matches_limb_convolution(N):
    rng = np.random.default_rng(N + 1)
    for a in (rng.integers(-256, 256, N), rng.integers(-(2**31), 2**31, N)):
        b = rand_u64(rng, N)
        assert np.array_equal(orc.poly_mul64(a, b), limb_negacyclic64(a, b))


@pytest.mark.parametrize("N", [8, 512, 2048])
def test_rotation64_identities(N):
    rng = np.random.default_rng(N + 9)
    p = rand_u64(rng, N)
    neg = np.uint64(0) - p
    assert np.array_equal(orc.rotate64(p, 0), p)
    assert np.array_equal(orc.rotate64(p, N), neg)                  # X^N = -1
    assert np.array_equal(orc.rotate64(orc.rotate64(p, N), N), p)   # X^{2N} = 1
    for _ in range(20):
        a, b = (int(x) for x in rng.integers(0, 2 * N, 2))
        assert np.array_equal(orc.rotate64(orc.rotate64(p, a), b), orc.rotate64(p, (a + b) % (2 * N)))
    for k in (1, 3, N - 1, N + 1, 2 * N - 1):
        mono = np.zeros(N, np.int64)
        mono[k % N] = 1 if k < N else -1
        assert np.array_equal(orc.rotate64(p, k), limb_negacyclic64(mono, p))


# ---- rounding steps ------------------------------------------------------------------

def brute_decompose64(t, l, Bgbit):
    """Balanced base-Bg digits of t rounded to l*Bgbit bits (independent route)."""
    shift = 64 - l * Bgbit
    r = ((t + (1 << (shift - 1))) >> shift) % (1 << (l * Bgbit))
    Bg = 1 << Bgbit
    digits, carry = [], 0
    for _ in range(l):
        d = (r & (Bg - 1)) + carry
        r >>= Bgbit
        carry = 1 if d >= Bg // 2 else 0
        digits.append(d - Bg if carry else d)
    return digits[::-1]


def test_decompose64_matches_balanced_base_conversion():
    rng = np.random.default_rng(22)
    l, Bgbit = 4, 9
    special = [0, 1, (1 << 27) - 1, 1 << 27, 1 << 28, 1 << 55, (1 << 63), M64, M64 - (1 << 27)]
    values = special + [int(x) for x in rand_u64(rng, 20000)]
    for t in values:
        d = orc.decompose64(l, Bgbit, t).tolist()
        assert d == brute_decompose64(t, l, Bgbit), t
        assert all(-256 <= x < 256 for x in d)
        rec = sum(x << (64 - (j + 1) * Bgbit) for j, x in enumerate(d))
        assert abs(s64(rec - t)) <= 1 << 27                          # half of 2^{64 - 36}
    assert orc.decompose64(l, Bgbit, 0).tolist() == [0, 0, 0, 0]


def test_pks_digits_round_to_t_digits():
    rng = np.random.default_rng(23)
    t, bb = 10, 3
    unit = 64 - t * bb                                              # 2^34
    special = [0, (1 << (unit - 1)) - 1, 1 << (unit - 1), 1 << unit, M64, 1 << 63]
    for a in special + [int(x) for x in rand_u64(rng, 20000)]:
        v = orc.pks_digits(t, bb, a).tolist()
        assert all(0 <= x < 8 for x in v)
        rec = sum(x << (64 - (j + 1) * bb) for j, x in enumerate(v)) & M64
        assert rec == (((a + (1 << (unit - 1))) >> unit) << unit) & M64, a


# ---- external product and CMUX over Torus64 ---------------------------------------

def gadget_trgsw64(N, l, Bgbit, m):
    C = np.zeros((2 * l, 2, N), np.uint64)
    for j in range(l):
        C[j, 0, 0] = (m << (64 - (j + 1) * Bgbit)) & M64
        C[l + j, 1, 0] = (m << (64 - (j + 1) * Bgbit)) & M64
    return C


def test_external_product64_brute_force_tiny():
    N, l, Bgbit = 8, 4, 9
    rng = np.random.default_rng(24)
    for _ in range(4):
        C = rand_u64(rng, (2 * l, 2, N))
        d = rand_u64(rng, (2, N))
        out = [[0] * N for _ in range(2)]
        for c in range(2):
            digs = [brute_decompose64(int(x), l, Bgbit) for x in d[c]]
            for j in range(l):
                poly = [dg[j] for dg in digs]
                for col in range(2):
                    prod = brute_negacyclic64(poly, C[c * l + j, col])
                    out[col] = [(x + y) % 2**64 for x, y in zip(out[col], prod)]
        assert orc.external_product64(l, Bgbit, C, d).tolist() == out


def test_external_product64_with_gadget_recomposes_and_cmux_selects():
    N, l, Bgbit = 64, 4, 9
    rng = np.random.default_rng(25)
    d = rand_u64(rng, (2, N))
    out = orc.external_product64(l, Bgbit, gadget_trgsw64(N, l, Bgbit, 1), d)
    err = [s64(int(x) - int(y)) for x, y in zip(d.reshape(-1), out.reshape(-1))]
    assert max(abs(e) for e in err) <= 1 << 27
    assert not orc.external_product64(l, Bgbit, gadget_trgsw64(N, l, Bgbit, 0), d).any()
    d1, d0 = rand_u64(rng, (2, N)), rand_u64(rng, (2, N))
    assert np.array_equal(orc.cmux64(l, Bgbit, gadget_trgsw64(N, l, Bgbit, 0), d1, d0), d0)
    sel = orc.cmux64(l, Bgbit, gadget_trgsw64(N, l, Bgbit, 1), d1, d0)
    assert max(abs(s64(int(x) - int(y))) for x, y in zip(sel.reshape(-1), d1.reshape(-1))) <= 1 << 27


# ---- BlindRotate, SampleExtract over the lvl2 ring -------------------------------------

def test_blind_rotate64_every_phase_tiny():
    """Noiseless BSK2, n=4, N2=16: the accumulator's phase is mu X^{-phi} sum_j X^j up to
    n (N2+1) decomposition roundings of 2^27, for every phi in Z_{2 N2}."""
    p = ti.Params(n=4, N=16, l=3, Bgbit=6, ks_t=5, ks_basebit=2, sigma0=0.0, sigma1=0.0)
    q = ti.CBParams(N2=16, l2=4, Bg2bit=9, pks_t=10, pks_basebit=3, sigma2=0.0, sigma_pks=0.0)
    s0 = np.array([1, 0, 1, 1], np.uint32)
    s2 = ti.keygen2(q, 31)
    bsk2 = ti.make_bsk2(p, q, 31, s0, s2)
    M = 2 * q.N2
    mu = 1 << 57
    bound = p.n * (q.N2 + 1) * (1 << 27)
    rng = np.random.default_rng(26)
    for phi in range(M):
        a = rng.integers(0, M, p.n)
        b = (phi + int((a * s0).sum())) % M
        acc = orc.blind_rotate64(p, q, bsk2, np.concatenate([a, [b]]).astype(np.uint32), mu)
        ph = orc.trlwe2_phase(s2, acc)
        for j in range(q.N2):
            expect = mu if (j + phi) % M < q.N2 else -mu
            assert abs(s64(int(ph[j]) - expect)) <= bound, (phi, j)


def test_sample_extract64_phase_is_coefficient_zero():
    rng = np.random.default_rng(27)
    for N in (8, 512, 2048):
        s = rng.integers(0, 2, N).astype(np.uint32)
        c = rand_u64(rng, (2, N))
        assert orc.tlwe2_phase(s, orc.sample_extract64(c)) == int(orc.trlwe2_phase(s, c)[0])


def test_cb_tlwe2_encrypts_m_over_bg_u():
    b = ti.cb_batch(ti.TOY, ti.CB_TOY, R=4)
    p, q = ti.TOY, ti.CB_TOY
    assert set(b.bits.tolist()) == {0, 1}
    for r in range(4):
        for u in (1, 2, 3):
            t2 = orc.cb_tlwe2(p, q, b.cbk.bsk2, b.tlwe[r], u)
            ph = orc.tlwe2_phase(b.cbk.s2, t2)
            expect = int(b.bits[r]) << (64 - u * p.Bgbit)
            assert abs(s64(ph - expect)) < 1 << 40, (r, u)


# ---- private functional key switching --------------------------------------------------

def test_private_keyswitch_noiseless_rounding_bound():
    """Noiseless PKSK: f_1 gives the input phase rounded to Torus32, f_0 gives -s1[X]
    times it, each within (N2+1) roundings of 2^{64-31} (2 Torus32 units) plus one."""
    p = ti.Params(n=4, N=32, l=3, Bgbit=6, ks_t=5, ks_basebit=2, sigma0=0.0, sigma1=0.0)
    q = ti.CBParams(N2=64, l2=4, Bg2bit=9, pks_t=10, pks_basebit=3, sigma2=0.0, sigma_pks=0.0)
    rng = np.random.default_rng(28)
    s1 = rng.integers(0, 2, p.N).astype(np.uint32)
    s2 = rng.integers(0, 2, q.N2).astype(np.uint32)
    pksk = ti.make_pksk(p, q, 41, s1, s2)
    bound = (q.N2 + 1) * 2 + 1
    for _ in range(6):
        c = rand_u64(rng, q.N2 + 1)
        x = ((orc.tlwe2_phase(s2, c) + (1 << 31)) >> 32) & M32        # phase rounded to Torus32
        ph1 = orc.trlwe_phase(s1, orc.private_keyswitch(p, q, pksk, 1, c))
        assert abs(s32(int(ph1[0]) - x)) <= bound
        assert all(abs(s32(int(v))) <= bound for v in ph1[1:])
        ph0 = orc.trlwe_phase(s1, orc.private_keyswitch(p, q, pksk, 0, c))
        for k in range(p.N):
            assert abs(s32(int(ph0[k]) + x * int(s1[k]))) <= bound, k


# ---- circuit bootstrapping end to end ---------------------------------------------------

@pytest.fixture(scope="module")
def cb_toy():
    b = ti.cb_batch(ti.TOY, ti.CB_TOY, R=4)
    return b, orc.circuit_bootstrap(ti.TOY, ti.CB_TOY, b.cbk.bsk2, b.cbk.pksk, b.tlwe)


def test_circuit_bootstrap_rows_decrypt(cb_toy):
    """Row u-1 has phase -m s1[X] / Bg^u and row l+u-1 has phase m / Bg^u (the TRGSW
    definition, Section 2.1.2), within 2^14 Torus32 units."""
    b, trgsw = cb_toy
    p = ti.TOY
    s1 = b.keys.s1.astype(np.int64)
    for r in range(len(b.bits)):
        m = int(b.bits[r])
        for row in range(2 * p.l):
            g = 1 << (32 - (row % p.l + 1) * p.Bgbit)
            if row < p.l:
                expect = (-m * g * s1) % 2**32
            else:
                expect = np.zeros(p.N, np.int64)
                expect[0] = m * g
            ph = orc.trlwe_phase(b.keys.s1, trgsw[r, row]).astype(np.int64)
            err = ((ph - expect + 2**31) % 2**32) - 2**31
            assert np.abs(err).max() < 1 << 14, (r, row)


def test_circuit_bootstrapped_trgsw_drives_cmux(cb_toy):
    b, trgsw = cb_toy
    p = ti.TOY
    rng = np.random.default_rng(29)
    m1 = rng.integers(0, 2, (1, p.N)).astype(np.uint8)
    m0 = rng.integers(0, 2, (1, p.N)).astype(np.uint8)
    d1 = ti.encrypt_trlwe_bits(p, 77, 1, b.keys.s1, m1)[0]
    d0 = ti.encrypt_trlwe_bits(p, 77, 2, b.keys.s1, m0)[0]
    for r in range(len(b.bits)):
        got = orc.trlwe_decrypt(b.keys.s1, orc.cmux(p, trgsw[r], d1, d0))
        assert np.array_equal(got, (m1 if b.bits[r] else m0)[0]), r


def test_cmux_tree_with_circuit_bootstrapped_address():
    """TLWE address bits -> circuit bootstrapping -> CMUX tree (Section 8.2: the memory
    controller feeds TLWE addresses, circuit bootstrapping makes them TRGSW)."""
    p, q = ti.TOY, ti.CB_TOY
    rom = ti.cmux_rom(p, ti.SEED_CB, v=3, R=2, packed=p.N)
    k = rom.keys
    for r in range(2):
        bits = ((int(rom.addrs[r]) >> np.arange(3)) & 1).astype(np.uint8)
        tl = ti.encrypt_tlwe0_bits(p, ti.SEED_CB, 95 + r, k.s0, bits)
        cbk = ti.cb_keys(p, q, ti.SEED_CB)
        addr = orc.circuit_bootstrap(p, q, cbk.bsk2, cbk.pksk, tl)
        out = orc.cmux_tree_read(p, addr, rom.table, 3)
        assert np.array_equal(orc.trlwe_decrypt(k.s1, out), rom.table_bits[rom.addrs[r]])


# ---- key sizes printed by the paper -------------------------------------------------------

def test_bootstrapping_key_size_matches_paper_table():
    rows = read_golden("key_sizes.txt")
    prm = {r[1]: int(r[2]) for r in rows if r[0] == "param"}
    printed = float([r for r in rows if r[0] == "printed_MB"][0][1])
    p = ti.Params(n=prm["n"], N=prm["N"], l=prm["l"], Bgbit=10, ks_t=prm["ks_t"],
                  ks_basebit=prm["ks_basebit"], sigma0=0.0, sigma1=0.0)
    q = ti.CBParams(N2=prm["N2"], l2=prm["l2"], Bg2bit=9, pks_t=prm["pks_t"],
                    pks_basebit=prm["pks_basebit"], sigma2=0.0, sigma_pks=0.0)
    bsk01 = p.n * 2 * p.l * 2 * p.N * 8
    iks = p.N * p.ks_t * (p.ks_base - 1) * (p.n + 1) * 4
    bsk02 = int(np.prod(ti.bsk2_shape(p, q))) * 8
    sh = ti.pksk_shape(p, q)                      # [2][N2+1][t][base][2][N]
    pks = sh[0] * sh[1] * sh[2] * (sh[3] - 1) * sh[4] * sh[5] * 4
    total = bsk01 + iks + bsk02 + pks
    assert round(total / 1e6, 3) == printed
