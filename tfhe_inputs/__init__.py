"""Seeded synthetic inputs for the TFHE gate-bootstrapping path.

This module only draws random numbers and performs the client-side encryptions
(keys, BSK, KSK, TLWE/TRLWE/TRGSW ciphertexts) that produce the evaluator's
inputs, plus the synthetic workloads (gate types, wiring, circuits, addresses).
It contains none of the evaluated arithmetic (no gate, CMUX, external product,
bootstrap, sample extraction or key switch), so the CPU oracle and the CUDA
library consume the same bytes without sharing code.

The paper (Section 2.1.2, "Parameters of TFHE") prints no parameter values; the
two parameter sets below are the toy set and the TFHE-like set of the workloads
this project measures.
"""
from __future__ import annotations

import ctypes
import dataclasses
import functools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfhe_inputs.c")
_LIB = os.path.join(_HERE, "libtfhe_inputs.so")

MU = 1 << 29  # 1/8 in Torus32


@dataclasses.dataclass(frozen=True)
class Params:
    n: int          # lvl0 TLWE dimension
    N: int          # lvl1 ring degree (power of two)
    l: int          # gadget levels
    Bgbit: int      # log2 of the gadget base Bg
    ks_t: int       # key-switching levels
    ks_basebit: int # log2 of the key-switching base
    sigma0: float   # lvl0 noise stdev (torus units)
    sigma1: float   # lvl1 noise stdev (torus units)

    @property
    def ks_base(self) -> int:
        return 1 << self.ks_basebit

    def abi(self):
        return (self.n, self.N, self.l, self.Bgbit, self.ks_t, self.ks_basebit)


# Toy (insecure) parameters: n=64, N=256, l=3, Bgbit=6, t=5, basebit=2.
TOY = Params(n=64, N=256, l=3, Bgbit=6, ks_t=5, ks_basebit=2, sigma0=2.0**-20, sigma1=2.0**-30)
# TFHE-like parameters: n=630, N=1024, l=3, Bgbit=6, t=8, basebit=2.
STD = Params(n=630, N=1024, l=3, Bgbit=6, ks_t=8, ks_basebit=2, sigma0=2.0**-15, sigma1=2.0**-25)

# Master seeds, one per workload family.
SEED_TOY = 0x20100941 + 1
SEED_FLAT = 0x20100941 + 2
SEED_DAG = 0x20100941 + 3
SEED_CMUX = 0x20100941 + 4
SEED_MIXED = 0x20100941 + 5
SEED_CB = 0x20100941 + 6


@dataclasses.dataclass(frozen=True)
class CBParams:
    """Circuit-bootstrapping parameters: the level-2 ring over the 64-bit torus and the
    private functional key switch back to lvl1 (the paper names circuit bootstrapping,
    Section 2.1.2, but prints no parameters)."""
    N2: int           # lvl2 ring degree
    l2: int           # lvl2 gadget levels
    Bg2bit: int       # log2 of the lvl2 gadget base
    pks_t: int        # private key-switching levels
    pks_basebit: int  # log2 of the private key-switching base
    sigma2: float     # lvl2 key noise stdev (Torus64 units)
    sigma_pks: float  # private key-switching key noise stdev (Torus32 units)

    @property
    def pks_base(self) -> int:
        return 1 << self.pks_basebit

    def abi(self):
        return (self.N2, self.l2, self.Bg2bit, self.pks_t, self.pks_basebit)


# lvl2 for the toy set (N2=512) and for the TFHE-like set (N2=2048); both l2=4, Bg2bit=9,
# private key switching t=10, basebit=3 (the sizes that reproduce the paper's "Size of Keys
# and Ciphertexts" table), with the lvl1 noise of the set.
CB_TOY = CBParams(N2=512, l2=4, Bg2bit=9, pks_t=10, pks_basebit=3, sigma2=2.0**-44,
                  sigma_pks=2.0**-30)
CB_STD = CBParams(N2=2048, l2=4, Bg2bit=9, pks_t=10, pks_basebit=3, sigma2=2.0**-44,
                  sigma_pks=2.0**-25)

GATE_NAMES = ["NAND", "AND", "OR", "NOR", "XOR", "XNOR", "ANDNY", "ANDYN", "ORNY", "ORYN"]


def plain_gate(t: int, a, b):
    """Plaintext truth function of gate type t (NY: first input negated)."""
    a = np.asarray(a).astype(bool)
    b = np.asarray(b).astype(bool)
    f = [
        lambda x, y: ~(x & y), lambda x, y: x & y, lambda x, y: x | y, lambda x, y: ~(x | y),
        lambda x, y: x ^ y, lambda x, y: ~(x ^ y), lambda x, y: ~x & y, lambda x, y: x & ~y,
        lambda x, y: ~x | y, lambda x, y: x | ~y,
    ][int(t)]
    return f(a, b).astype(np.uint8)


class _CParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("N", ctypes.c_int32), ("l", ctypes.c_int32),
                ("Bgbit", ctypes.c_int32), ("ks_t", ctypes.c_int32),
                ("ks_basebit", ctypes.c_int32), ("sigma0", ctypes.c_double),
                ("sigma1", ctypes.c_double)]


class _CCbParams(ctypes.Structure):
    _fields_ = [("N2", ctypes.c_int32), ("l2", ctypes.c_int32), ("Bg2bit", ctypes.c_int32),
                ("pks_t", ctypes.c_int32), ("pks_basebit", ctypes.c_int32),
                ("sigma2", ctypes.c_double), ("sigma_pks", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the generator into an in-tree shared library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-std=c11", "-fopenmp", "-o",
                               _LIB, _SRC, "-lm"])
    return _LIB


@functools.lru_cache(maxsize=1)
def _lib():
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.POINTER(_CParams)
    u32p = ctypes.c_void_p
    lib.tin_keygen.argtypes = [P, ctypes.c_uint64, u32p, u32p]
    lib.tin_bsk.argtypes = [P, ctypes.c_uint64, u32p, u32p, u32p]
    lib.tin_ksk.argtypes = [P, ctypes.c_uint64, u32p, u32p, u32p]
    for f in (lib.tin_tlwe0_encrypt_bits, lib.tin_trlwe_encrypt_bits, lib.tin_trgsw_encrypt_bits):
        f.argtypes = [P, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p, ctypes.c_int64, u32p]
    lib.tin_random_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, u32p]
    Q = ctypes.POINTER(_CCbParams)
    lib.tin_keygen2.argtypes = [Q, ctypes.c_uint64, u32p]
    lib.tin_bsk2.argtypes = [P, Q, ctypes.c_uint64, u32p, u32p, u32p]
    lib.tin_pksk.argtypes = [P, Q, ctypes.c_uint64, u32p, u32p, u32p]
    for f in (lib.tin_keygen, lib.tin_bsk, lib.tin_ksk, lib.tin_tlwe0_encrypt_bits,
              lib.tin_trlwe_encrypt_bits, lib.tin_trgsw_encrypt_bits, lib.tin_random_u64,
              lib.tin_keygen2, lib.tin_bsk2, lib.tin_pksk):
        f.restype = None
    return lib


def _cp(p: Params):
    return ctypes.byref(_CParams(p.n, p.N, p.l, p.Bgbit, p.ks_t, p.ks_basebit, p.sigma0, p.sigma1))


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _cq(q: CBParams):
    return ctypes.byref(_CCbParams(q.N2, q.l2, q.Bg2bit, q.pks_t, q.pks_basebit, q.sigma2,
                                   q.sigma_pks))


def keygen2(q: CBParams, seed: int) -> np.ndarray:
    """lvl2 key s2 in B_{N2}[X]."""
    s2 = np.zeros(q.N2, np.uint32)
    _lib().tin_keygen2(_cq(q), seed, _ptr(s2))
    return s2


def bsk2_shape(p: Params, q: CBParams):
    return (p.n, 2 * q.l2, 2, q.N2)


def pksk_shape(p: Params, q: CBParams):
    return (2, q.N2 + 1, q.pks_t, q.pks_base, 2, p.N)


def make_bsk2(p: Params, q: CBParams, seed: int, s0, s2) -> np.ndarray:
    """BSK2 u64[n][2 l2][2][N2]: TRGSW_{s2}(s0[i]) over Torus64."""
    bsk2 = np.zeros(bsk2_shape(p, q), np.uint64)
    _lib().tin_bsk2(_cp(p), _cq(q), seed, _ptr(s0), _ptr(s2), _ptr(bsk2))
    return bsk2


def make_pksk(p: Params, q: CBParams, seed: int, s1, s2) -> np.ndarray:
    """PKSK u32[2][N2+1][t][base][2][N]: private functional key-switching keys for
    f_0(x) = -s1[X] x and f_1(x) = x."""
    pksk = np.zeros(pksk_shape(p, q), np.uint32)
    _lib().tin_pksk(_cp(p), _cq(q), seed, _ptr(s1), _ptr(s2), _ptr(pksk))
    return pksk


def keygen(p: Params, seed: int):
    s0 = np.zeros(p.n, np.uint32)
    s1 = np.zeros(p.N, np.uint32)
    _lib().tin_keygen(_cp(p), seed, _ptr(s0), _ptr(s1))
    return s0, s1


def make_bsk(p: Params, seed: int, s0, s1) -> np.ndarray:
    bsk = np.zeros((p.n, 2 * p.l, 2, p.N), np.uint32)
    _lib().tin_bsk(_cp(p), seed, _ptr(s0), _ptr(s1), _ptr(bsk))
    return bsk


def make_ksk(p: Params, seed: int, s0, s1) -> np.ndarray:
    ksk = np.zeros((p.N, p.ks_t, p.ks_base, p.n + 1), np.uint32)
    _lib().tin_ksk(_cp(p), seed, _ptr(s0), _ptr(s1), _ptr(ksk))
    return ksk


def encrypt_tlwe0_bits(p: Params, seed: int, stream: int, s0, bits) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    out = np.zeros((bits.size, p.n + 1), np.uint32)
    _lib().tin_tlwe0_encrypt_bits(_cp(p), seed, stream, _ptr(s0), _ptr(bits), bits.size,
                                  _ptr(out))
    return out


def encrypt_trlwe_bits(p: Params, seed: int, stream: int, s1, msg) -> np.ndarray:
    msg = np.ascontiguousarray(msg, dtype=np.uint8).reshape(-1, p.N)
    out = np.zeros((msg.shape[0], 2, p.N), np.uint32)
    _lib().tin_trlwe_encrypt_bits(_cp(p), seed, stream, _ptr(s1), _ptr(msg), msg.shape[0],
                                  _ptr(out))
    return out


def encrypt_trgsw_bits(p: Params, seed: int, stream: int, s1, bits) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8).reshape(-1)
    out = np.zeros((bits.size, 2 * p.l, 2, p.N), np.uint32)
    _lib().tin_trgsw_encrypt_bits(_cp(p), seed, stream, _ptr(s1), _ptr(bits), bits.size,
                                  _ptr(out))
    return out


def random_u64(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.zeros(count, np.uint64)
    _lib().tin_random_u64(seed, stream, count, _ptr(out))
    return out


def random_bits(seed: int, stream: int, count: int) -> np.ndarray:
    return (random_u64(seed, stream, count) >> np.uint64(63)).astype(np.uint8)


def random_below(seed: int, stream: int, count: int, bound: int) -> np.ndarray:
    """Uniform integers in [0, bound) (multiply-shift on the high 32 bits)."""
    hi = random_u64(seed, stream, count) >> np.uint64(32)
    return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


# ---------------------------------------------------------------------------
# Keys (cached per process: the TFHE-like BSK takes a few seconds to encrypt)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Keys:
    params: Params
    s0: np.ndarray
    s1: np.ndarray
    bsk: np.ndarray
    ksk: np.ndarray


@functools.lru_cache(maxsize=4)
def keys(p: Params, seed: int) -> Keys:
    s0, s1 = keygen(p, seed)
    return Keys(p, s0, s1, make_bsk(p, seed, s0, s1), make_ksk(p, seed, s0, s1))


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class GateBatch:
    """One batch of independent gates: out[g] = gate(types[g], inp[idx[g,0]], inp[idx[g,1]])."""
    keys: Keys
    bits: np.ndarray      # u8[num_in] plaintext of the inputs
    inp: np.ndarray       # u32[num_in][n+1] TLWE lvl0
    types: np.ndarray     # u8[G]
    idx: np.ndarray       # i32[G][2]

    @property
    def expected(self) -> np.ndarray:
        return np.array([plain_gate(t, self.bits[a], self.bits[b])
                         for t, (a, b) in zip(self.types, self.idx)], np.uint8)


def toy_gates(seed: int = SEED_TOY, p: Params = TOY) -> GateBatch:
    """40 gates, 4 of each of the 10 types in enum order, on 80 random encrypted bits."""
    k = keys(p, seed)
    types = np.repeat(np.arange(10, dtype=np.uint8), 4)
    bits = random_bits(seed, 1, 2 * types.size)
    inp = encrypt_tlwe0_bits(p, seed, 1, k.s0, bits)
    idx = np.arange(2 * types.size, dtype=np.int32).reshape(-1, 2)
    return GateBatch(k, bits, inp, types, idx)


def flat_level(G: int = 4096, seed: int = SEED_FLAT, p: Params = STD) -> GateBatch:
    """One flat level of G independent gates, types uniform over the 10 gates,
    each gate reading its own two fresh encrypted random bits."""
    k = keys(p, seed)
    types = random_below(seed, 2, G, 10).astype(np.uint8)
    bits = random_bits(seed, 1, 2 * G)
    inp = encrypt_tlwe0_bits(p, seed, 1, k.s0, bits)
    idx = np.arange(2 * G, dtype=np.int32).reshape(-1, 2)
    return GateBatch(k, bits, inp, types, idx)


@dataclasses.dataclass
class Circuit:
    """A layered DAG: wire w < num_inputs is a primary input; wire num_inputs + g
    is the output of gate g.  Gates are listed in topological order."""
    num_inputs: int
    types: np.ndarray     # u8[G]
    idx: np.ndarray       # i32[G][2] wire indices
    level: np.ndarray     # i32[G] generation level (0-based)

    @property
    def num_gates(self) -> int:
        return int(self.types.size)

    def evaluate_plain(self, in_bits: np.ndarray) -> np.ndarray:
        w = np.zeros(self.num_inputs + self.num_gates, np.uint8)
        w[: self.num_inputs] = in_bits
        for g in range(self.num_gates):
            a, b = self.idx[g]
            w[self.num_inputs + g] = plain_gate(self.types[g], w[a], w[b])
        return w[self.num_inputs:]


def _widths(seed: int, stream: int, levels: int, total: int, lo: int, hi: int) -> np.ndarray:
    """Level widths: draw U[lo, hi] per level, scale to `total`, round by largest
    remainder, keep every width >= 1 (and within [lo, hi] when the total allows it)."""
    raw = lo + random_below(seed, stream, levels, hi - lo + 1)
    scaled = raw * (total / raw.sum())
    w = np.floor(scaled).astype(np.int64)
    rem = total - int(w.sum())
    order = np.argsort(-(scaled - w), kind="stable")
    w[order[:rem]] += 1
    w = np.maximum(w, 1)
    feasible = levels * lo <= total <= levels * hi
    if feasible:
        # clamp into [lo, hi] and move the excess/deficit to levels that have room
        for _ in range(8):
            over = np.maximum(w - hi, 0).sum()
            under = np.maximum(lo - w, 0).sum()
            w = np.clip(w, lo, hi)
            diff = over - under
            i = 0
            while diff != 0 and i < 100 * levels:
                j = i % levels
                if diff > 0 and w[j] < hi:
                    w[j] += 1; diff -= 1
                elif diff < 0 and w[j] > lo:
                    w[j] -= 1; diff += 1
                i += 1
    # fix any rounding drift
    d = total - int(w.sum())
    j = 0
    while d != 0:
        if d > 0:
            w[j % levels] += 1; d -= 1
        elif w[j % levels] > 1:
            w[j % levels] -= 1; d += 1
        j += 1
    return w


def layered_dag(seed: int = SEED_DAG, total: int = 20000, levels: int = 60,
                num_inputs: int = 256, lo: int = 50, hi: int = 800, stream: int = 0) -> Circuit:
    """Random layered DAG: level widths U[lo,hi] scaled to `total`; each gate input is
    drawn uniformly from the outputs of the previous 3 levels and the primaries."""
    w = _widths(seed, 100 + stream, levels, total, lo, hi)
    G = int(w.sum())
    types = random_below(seed, 200 + stream, G, 10).astype(np.uint8)
    r = random_u64(seed, 300 + stream, 2 * G) >> np.uint64(32)
    idx = np.zeros((G, 2), np.int32)
    level = np.zeros(G, np.int32)
    starts = np.concatenate([[0], np.cumsum(w)])
    g = 0
    for L in range(levels):
        lo_lvl = max(0, L - 3)
        # candidate wires: primaries + outputs of levels lo_lvl..L-1
        cand_gate_lo = int(starts[lo_lvl])
        cand_gate_hi = int(starts[L])
        n_cand = num_inputs + (cand_gate_hi - cand_gate_lo)
        for _ in range(int(w[L])):
            for s in range(2):
                c = int((int(r[2 * g + s]) * n_cand) >> 32)
                idx[g, s] = c if c < num_inputs else num_inputs + cand_gate_lo + (c - num_inputs)
            level[g] = L
            g += 1
    return Circuit(num_inputs, types, idx, level)


def mixed_circuits(seed: int = SEED_MIXED, count: int = 16, gmin: int = 2000, gmax: int = 40000,
                   lmin: int = 20, lmax: int = 120, num_inputs: int = 256):
    """`count` independent layered circuits of uneven size and depth."""
    sizes = gmin + random_below(seed, 1, count, gmax - gmin + 1)
    depths = lmin + random_below(seed, 2, count, lmax - lmin + 1)
    return [layered_dag(seed, int(sizes[c]), int(depths[c]), num_inputs, 50, 800, stream=c + 1)
            for c in range(count)]


@dataclasses.dataclass
class CmuxRom:
    """A table of 2^v TRLWE rows read at R addresses given as encrypted TRGSW bits."""
    keys: Keys
    v: int
    table_bits: np.ndarray   # u8[2^v][N] plaintext (bits in coefficients 0..packed-1)
    table: np.ndarray        # u32[2^v][2][N]
    addrs: np.ndarray        # i64[R]
    addr_trgsw: np.ndarray   # u32[R][v][2l][2][N], bit j of the address at [r][j]


def cmux_rom(p: Params = STD, seed: int = SEED_CMUX, v: int = 9, R: int = 64,
             packed: int = 32) -> CmuxRom:
    """Table of 2^v rows each packing `packed` random bits in coefficients 0..packed-1
    (other coefficients encode 0), read at R distinct random addresses."""
    k = keys(p, seed)
    rows = 1 << v
    tb = np.zeros((rows, p.N), np.uint8)
    tb[:, :packed] = random_bits(seed, 10, rows * packed).reshape(rows, packed)
    table = encrypt_trlwe_bits(p, seed, 10, k.s1, tb)
    perm = np.argsort(random_u64(seed, 11, rows), kind="stable")
    addrs = perm[:R].astype(np.int64)
    abits = ((addrs[:, None] >> np.arange(v)[None, :]) & 1).astype(np.uint8)
    addr_trgsw = encrypt_trgsw_bits(p, seed, 12, k.s1, abits.reshape(-1)).reshape(
        R, v, 2 * p.l, 2, p.N)
    return CmuxRom(k, v, tb, table, addrs, addr_trgsw)


@dataclasses.dataclass
class RamWrite:
    keys: Keys
    v: int
    cell_bits: np.ndarray   # u8[2^v][N]
    cells: np.ndarray       # u32[2^v][2][N]
    new_bits: np.ndarray    # u8[N]
    new_cell: np.ndarray    # u32[2][N]
    addr: int
    addr_trgsw: np.ndarray  # u32[v][2l][2][N]


def ram_write(p: Params = STD, seed: int = SEED_CMUX, v: int = 8, packed: int = 32) -> RamWrite:
    """A RAM of 2^v TRLWE cells, a new cell and a random encrypted address."""
    k = keys(p, seed)
    cells_n = 1 << v
    cb = np.zeros((cells_n, p.N), np.uint8)
    cb[:, :packed] = random_bits(seed, 20, cells_n * packed).reshape(cells_n, packed)
    cells = encrypt_trlwe_bits(p, seed, 20, k.s1, cb)
    nb = np.zeros((1, p.N), np.uint8)
    nb[0, :packed] = random_bits(seed, 21, packed)
    new_cell = encrypt_trlwe_bits(p, seed, 21, k.s1, nb)[0]
    addr = int(random_below(seed, 22, 1, cells_n)[0])
    abits = ((addr >> np.arange(v)) & 1).astype(np.uint8)
    addr_trgsw = encrypt_trgsw_bits(p, seed, 23, k.s1, abits)
    return RamWrite(k, v, cb, cells, nb[0], new_cell, addr, addr_trgsw)


@dataclasses.dataclass
class RamCycle:
    keys: Keys
    v: int
    w: int
    cell_bits: np.ndarray   # u8[w][2^v]: bit of word x in block b at [b][x]
    cells: np.ndarray       # u32[w][2^v][2][N], the bit at coefficient 0
    addr: int
    addr_trgsw: np.ndarray  # u32[v][2l][2][N]
    flag_bit: int
    flag: np.ndarray        # u32[n+1]
    wdata_bits: np.ndarray  # u8[w]
    wdata: np.ndarray       # u32[w][n+1]


def ram_cycle(p: Params = STD, seed: int = SEED_CMUX, v: int = 8, w: int = 16,
              flag_bit: int = 1, stream: int = 0) -> RamCycle:
    """A RAM of 2^v words of w bits (one TRLWE per bit, the bit at coefficient 0, the
    other coefficients encoding 0), a random encrypted address, write flag and word."""
    k = keys(p, seed)
    rows = 1 << v
    cb = random_bits(seed, 70 + stream, w * rows).reshape(w, rows)
    msg = np.zeros((w * rows, p.N), np.uint8)
    msg[:, 0] = cb.reshape(-1)
    cells = encrypt_trlwe_bits(p, seed, 70 + stream, k.s1, msg).reshape(w, rows, 2, p.N)
    addr = int(random_below(seed, 71 + stream, 1, rows)[0])
    abits = ((addr >> np.arange(v)) & 1).astype(np.uint8)
    addr_trgsw = encrypt_trgsw_bits(p, seed, 72 + stream, k.s1, abits)
    flag = encrypt_tlwe0_bits(p, seed, 73 + stream, k.s0, np.array([flag_bit], np.uint8))[0]
    wb = random_bits(seed, 74 + stream, w)
    wdata = encrypt_tlwe0_bits(p, seed, 75 + stream, k.s0, wb)
    return RamCycle(k, v, w, cb, cells, addr, addr_trgsw, flag_bit, flag, wb, wdata)


@dataclasses.dataclass
class PackedRom:
    keys: Keys
    v: int
    w: int
    words: np.ndarray       # u8[M][w] plaintext bits
    table: np.ndarray       # u32[T][2][N]: word q of TRLWE t at coefficients q w .. q w + w - 1
    addrs: np.ndarray       # i64[R]
    addr_trgsw: np.ndarray  # u32[R][v][2l][2][N]


def packed_rom(p: Params = STD, seed: int = SEED_CMUX, M: int = 128, w: int = 32,
               R: int = 8, stream: int = 0) -> PackedRom:
    """ROM of M words of w bits with vertical and horizontal packing (N / w words per
    TRLWE), read at R random addresses."""
    k = keys(p, seed)
    P = p.N // w
    T = M // P
    v = int(M).bit_length() - 1
    words = random_bits(seed, 80 + stream, M * w).reshape(M, w)
    msg = words.reshape(T, P * w)
    table = encrypt_trlwe_bits(p, seed, 80 + stream, k.s1, msg)
    addrs = random_below(seed, 81 + stream, R, M).astype(np.int64)
    abits = ((addrs[:, None] >> np.arange(v)[None, :]) & 1).astype(np.uint8)
    addr_trgsw = encrypt_trgsw_bits(p, seed, 82 + stream, k.s1, abits.reshape(-1)).reshape(
        R, v, 2 * p.l, 2, p.N)
    return PackedRom(k, v, w, words, table, addrs, addr_trgsw)


@dataclasses.dataclass
class CBKeys:
    s2: np.ndarray    # u32[N2] lvl2 key
    bsk2: np.ndarray  # u64[n][2 l2][2][N2]
    pksk: np.ndarray  # u32[2][N2+1][t][base][2][N]


@functools.lru_cache(maxsize=2)
def cb_keys(p: Params, q: CBParams, seed: int) -> CBKeys:
    k = keys(p, seed)
    s2 = keygen2(q, seed)
    return CBKeys(s2, make_bsk2(p, q, seed, k.s0, s2), make_pksk(p, q, seed, k.s1, s2))


@dataclasses.dataclass
class CBBatch:
    keys: Keys
    cbk: CBKeys
    bits: np.ndarray  # u8[R]
    tlwe: np.ndarray  # u32[R][n+1] lvl0 encryptions of bits


def cb_batch(p: Params = TOY, q: CBParams = CB_TOY, seed: int = SEED_CB, R: int = 4,
             stream: int = 0) -> CBBatch:
    """R lvl0 TLWE encryptions of uniform random bits to circuit-bootstrap."""
    k = keys(p, seed)
    bits = random_bits(seed, 90 + stream, R)
    return CBBatch(k, cb_keys(p, q, seed), bits, encrypt_tlwe0_bits(p, seed, 90 + stream, k.s0,
                                                                      bits))
