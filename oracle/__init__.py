"""CPU oracle for TFHE gate bootstrapping and CMUX memory (test infrastructure only).

A thin ctypes wrapper over `tfhe_oracle.c`, a plain schoolbook implementation of
the scheme's definitions (paper Section 2.1.2 "TFHE" and Section 8 "CMUX Memory").
Only the tests, the smoke check and the CPU-baseline leg of the benchmark import
this package; the product library never does, and this package imports nothing
from the product library.

Every function is written against the definitions; all arithmetic is mod 2^32, except
the level-2 ring of circuit bootstrapping (reading R16), which is mod 2^64.
Parity of absolute ciphertext words with the CUDA path rests on the readings R1-R8
listed at the top of `tfhe_oracle.c`; those readings are pinned by the properties
the scheme fixes (decryption, truth tables, rounding bounds, algebraic
identities, structure counts), not by printed ciphertexts (the paper prints none).
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfhe_oracle.c")
_LIB = os.path.join(_HERE, "libtfhe_oracle.so")


class _P(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("N", ctypes.c_int32), ("l", ctypes.c_int32),
                ("Bgbit", ctypes.c_int32), ("ks_t", ctypes.c_int32),
                ("ks_basebit", ctypes.c_int32)]


class _Q(ctypes.Structure):
    _fields_ = [("N2", ctypes.c_int32), ("l2", ctypes.c_int32), ("Bg2bit", ctypes.c_int32),
                ("pks_t", ctypes.c_int32), ("pks_basebit", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-std=c11", "-o", _LIB, _SRC])
    return _LIB


@functools.lru_cache(maxsize=1)
def _lib():
    build()
    lib = ctypes.CDLL(_LIB)
    vp, i32, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32
    P = ctypes.POINTER(_P)
    Q = ctypes.POINTER(_Q)
    sig = {
        "orc_poly_mul": (None, [i32, vp, vp, vp]),
        "orc_rotate": (None, [i32, i32, vp, vp]),
        "orc_tlwe_phase": (u32, [i32, vp, vp]),
        "orc_tlwe_decrypt": (i32, [i32, vp, vp]),
        "orc_trlwe_phase": (None, [i32, vp, vp, vp]),
        "orc_trlwe_decrypt": (None, [i32, vp, vp, vp]),
        "orc_decompose": (None, [i32, i32, u32, vp]),
        "orc_external_product": (None, [P, vp, vp, vp]),
        "orc_cmux": (None, [P, vp, vp, vp, vp]),
        "orc_modswitch": (u32, [i32, u32]),
        "orc_ks_digits": (None, [i32, i32, u32, vp]),
        "orc_blind_rotate": (None, [P, vp, vp, vp]),
        "orc_sample_extract": (None, [i32, vp, vp]),
        "orc_keyswitch": (None, [P, vp, vp, vp]),
        "orc_gate_combine": (i32, [i32, i32, vp, vp, vp]),
        "orc_homgate": (i32, [P, vp, vp, i32, vp, vp, vp]),
        "orc_gate_batch": (i32, [P, vp, vp, vp, ctypes.c_int64, vp, vp, vp, ctypes.c_int64,
                                 ctypes.c_int64]),
        "orc_hommux_noks": (None, [P, vp, vp, vp, vp, vp]),
        "orc_hommux": (None, [P, vp, vp, vp, vp, vp, vp]),
        "orc_mux_batch": (i32, [P, vp, vp, vp, ctypes.c_int64, vp, i32, vp, ctypes.c_int64,
                                ctypes.c_int64]),
        "orc_cmux_tree_read": (None, [P, vp, vp, i32, vp]),
        "orc_ram_cycle": (None, [P, vp, vp, vp, i32, i32, vp, vp, vp, vp]),
        "orc_rom_read": (None, [P, vp, vp, vp, i32, i32, vp, vp]),
        "orc_ram_write": (None, [P, vp, i32, vp, vp]),
        "orc64_poly_mul": (None, [i32, vp, vp, vp]),
        "orc64_rotate": (None, [i32, i32, vp, vp]),
        "orc64_tlwe_phase": (ctypes.c_uint64, [i32, vp, vp]),
        "orc64_trlwe_phase": (None, [i32, vp, vp, vp]),
        "orc64_decompose": (None, [i32, i32, ctypes.c_uint64, vp]),
        "orc64_external_product": (None, [i32, i32, i32, vp, vp, vp]),
        "orc64_cmux": (None, [i32, i32, i32, vp, vp, vp, vp]),
        "orc64_blind_rotate": (None, [P, Q, vp, vp, ctypes.c_uint64, vp]),
        "orc64_sample_extract": (None, [i32, vp, vp]),
        "orc_cb_tlwe2": (None, [P, Q, vp, vp, i32, vp]),
        "orc_pks_digits": (None, [i32, i32, ctypes.c_uint64, vp]),
        "orc_private_keyswitch": (None, [P, Q, vp, i32, vp, vp]),
        "orc_circuit_bootstrap": (None, [P, Q, vp, vp, vp, vp]),
        "orc_extprod_count": (ctypes.c_uint64, []),
        "orc_extprod_count_reset": (None, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _p(params):
    n, N, l, Bgbit, t, bb = params.abi() if hasattr(params, "abi") else params
    return ctypes.byref(_P(n, N, l, Bgbit, t, bb))


def _q(cbp):
    return ctypes.byref(_Q(*cbp.abi()))


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data)


# ---- polynomial primitives -----------------------------------------------------

def poly_mul(a_int, b_torus):
    a, pa = _c(a_int, np.int32)
    b, pb = _c(b_torus, np.uint32)
    out = np.zeros(a.size, np.uint32)
    _lib().orc_poly_mul(a.size, pa, pb, ctypes.c_void_p(out.ctypes.data))
    return out


def rotate(p, k):
    a, pa = _c(p, np.uint32)
    out = np.zeros(a.size, np.uint32)
    _lib().orc_rotate(a.size, int(k), pa, ctypes.c_void_p(out.ctypes.data))
    return out


def decompose(l, Bgbit, t):
    out = np.zeros(l, np.int32)
    _lib().orc_decompose(l, Bgbit, int(t) & 0xFFFFFFFF, ctypes.c_void_p(out.ctypes.data))
    return out


def ks_digits(t, basebit, a):
    out = np.zeros(t, np.uint32)
    _lib().orc_ks_digits(t, basebit, int(a) & 0xFFFFFFFF, ctypes.c_void_p(out.ctypes.data))
    return out


def fn_address(name: str) -> int:
    """Address of an oracle C function (for the exhaustive C checkers in the tests)."""
    return ctypes.cast(getattr(_lib(), name), ctypes.c_void_p).value


def modswitch(N, x):
    return int(_lib().orc_modswitch(N, int(x) & 0xFFFFFFFF))


# ---- encryption-side checks ------------------------------------------------------

def tlwe_phase(s, c):
    s, ps = _c(s, np.uint32)
    c, pc = _c(c, np.uint32)
    return int(_lib().orc_tlwe_phase(s.size, ps, pc))


def tlwe_decrypt(s, c) -> np.ndarray:
    """Decrypt one TLWE (u32[n+1]) or a batch (u32[k][n+1])."""
    s, ps = _c(s, np.uint32)
    c = np.ascontiguousarray(c, np.uint32)
    flat = c.reshape(-1, s.size + 1)
    out = np.array([_lib().orc_tlwe_decrypt(s.size, ps, ctypes.c_void_p(row.ctypes.data))
                    for row in flat], np.uint8)
    return out if c.ndim > 1 else out[0]


def trlwe_phase(s, c):
    s, ps = _c(s, np.uint32)
    c, pc = _c(c, np.uint32)
    out = np.zeros(s.size, np.uint32)
    _lib().orc_trlwe_phase(s.size, ps, pc, ctypes.c_void_p(out.ctypes.data))
    return out


def trlwe_decrypt(s, c):
    s, ps = _c(s, np.uint32)
    c, pc = _c(c, np.uint32)
    out = np.zeros(s.size, np.uint8)
    _lib().orc_trlwe_decrypt(s.size, ps, pc, ctypes.c_void_p(out.ctypes.data))
    return out


# ---- evaluation ----------------------------------------------------------------

def external_product(params, C, d):
    C, pC = _c(C, np.uint32)
    d, pd = _c(d, np.uint32)
    out = np.zeros_like(d)
    _lib().orc_external_product(_p(params), pC, pd, ctypes.c_void_p(out.ctypes.data))
    return out


def cmux(params, C, d1, d0):
    C, pC = _c(C, np.uint32)
    d1, p1 = _c(d1, np.uint32)
    d0, p0 = _c(d0, np.uint32)
    out = np.zeros_like(d0)
    _lib().orc_cmux(_p(params), pC, p1, p0, ctypes.c_void_p(out.ctypes.data))
    return out


def blind_rotate(params, bsk, bar):
    bsk, pb = _c(bsk, np.uint32)
    bar, pbar = _c(bar, np.uint32)
    out = np.zeros((2, params.N), np.uint32)
    _lib().orc_blind_rotate(_p(params), pb, pbar, ctypes.c_void_p(out.ctypes.data))
    return out


def sample_extract(trlwe):
    c, pc = _c(trlwe, np.uint32)
    N = c.shape[-1]
    out = np.zeros(N + 1, np.uint32)
    _lib().orc_sample_extract(N, pc, ctypes.c_void_p(out.ctypes.data))
    return out


def keyswitch(params, ksk, tlwe1):
    k, pk = _c(ksk, np.uint32)
    c, pc = _c(tlwe1, np.uint32)
    out = np.zeros(params.n + 1, np.uint32)
    _lib().orc_keyswitch(_p(params), pk, pc, ctypes.c_void_p(out.ctypes.data))
    return out


def gate_combine(n, gate_type, c1, c2):
    a, pa = _c(c1, np.uint32)
    b, pb = _c(c2, np.uint32)
    out = np.zeros(n + 1, np.uint32)
    rc = _lib().orc_gate_combine(n, int(gate_type), pa, pb, ctypes.c_void_p(out.ctypes.data))
    if rc != 0:
        raise ValueError("unknown gate type")
    return out


def homgate(params, bsk, ksk, gate_type, c1, c2):
    bsk, pb = _c(bsk, np.uint32)
    ksk, pk = _c(ksk, np.uint32)
    a, pa = _c(c1, np.uint32)
    b, pbb = _c(c2, np.uint32)
    out = np.zeros(params.n + 1, np.uint32)
    rc = _lib().orc_homgate(_p(params), pb, pk, int(gate_type), pa, pbb,
                            ctypes.c_void_p(out.ctypes.data))
    if rc != 0:
        raise ValueError("unknown gate type")
    return out


def gate_batch(params, bsk, ksk, inp, types, idx, gates=None, threads: int | None = None):
    """Evaluate gates (all, or the listed subset) of a batch; one gate per thread.

    Returns u32[len(gates)][n+1] in the order of `gates`."""
    bsk, pb = _c(bsk, np.uint32)
    ksk, pk = _c(ksk, np.uint32)
    inp, pi = _c(inp, np.uint32)
    types, pt = _c(types, np.uint8)
    idx, px = _c(idx, np.int32)
    G = types.size
    gates = np.arange(G) if gates is None else np.asarray(gates, np.int64)
    out = np.zeros((G, params.n + 1), np.uint32)
    po = ctypes.c_void_p(out.ctypes.data)
    pp = _p(params)
    lib = _lib()

    def one(g):
        rc = lib.orc_gate_batch(pp, pb, pk, pi, inp.shape[0], pt, px, po, int(g), int(g) + 1)
        if rc != 0:
            raise ValueError(f"bad gate {g}")

    threads = threads or os.cpu_count() or 1
    if threads == 1 or len(gates) == 1:
        for g in gates:
            one(g)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(one, gates))
    return out[gates]


def hommux_noks(params, bsk, c, a, b):
    """HomMUX without SE and IKS (reading R13): TLWE c, a, b -> TRLWE u32[2][N]."""
    bsk, pb = _c(bsk, np.uint32)
    (c, pc), (a, pa), (b, pbb) = _c(c, np.uint32), _c(a, np.uint32), _c(b, np.uint32)
    out = np.zeros((2, params.N), np.uint32)
    _lib().orc_hommux_noks(_p(params), pb, pc, pa, pbb, ctypes.c_void_p(out.ctypes.data))
    return out


def hommux(params, bsk, ksk, c, a, b):
    """HomMUX (reading R13): TLWE c, a, b -> TLWE u32[n+1] decrypting to c ? a : b."""
    bsk, pb = _c(bsk, np.uint32)
    ksk, pk = _c(ksk, np.uint32)
    (c, pc), (a, pa), (b, pbb) = _c(c, np.uint32), _c(a, np.uint32), _c(b, np.uint32)
    out = np.zeros(params.n + 1, np.uint32)
    _lib().orc_hommux(_p(params), pb, pk, pc, pa, pbb, ctypes.c_void_p(out.ctypes.data))
    return out


def mux_batch(params, bsk, ksk, inp, idx, noks=False, gates=None, threads: int | None = None):
    """MUXes of a batch (idx [G][3]: selector, input taken when it is 1, the other), all
    or the listed subset, one per thread.  TLWE outputs u32[*][n+1], or TRLWE outputs
    u32[*][2][N] with noks."""
    bsk, pb = _c(bsk, np.uint32)
    ksk, pk = _c(ksk, np.uint32)
    inp, pi = _c(inp, np.uint32)
    idx, px = _c(idx, np.int32)
    G = idx.shape[0]
    gates = np.arange(G) if gates is None else np.asarray(gates, np.int64)
    out = (np.zeros((G, 2, params.N), np.uint32) if noks
           else np.zeros((G, params.n + 1), np.uint32))
    po = ctypes.c_void_p(out.ctypes.data)
    pp = _p(params)
    lib = _lib()

    def one(g):
        if lib.orc_mux_batch(pp, pb, pk, pi, inp.shape[0], px, 1 if noks else 0, po,
                             int(g), int(g) + 1) != 0:
            raise ValueError(f"bad mux {g}")

    threads = threads or os.cpu_count() or 1
    if threads == 1 or len(gates) == 1:
        for g in gates:
            one(g)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(one, gates))
    return out[gates]


def cmux_tree_read(params, addr_trgsw, table, v):
    a, pa = _c(addr_trgsw, np.uint32)
    t, pt = _c(table, np.uint32)
    out = np.zeros((2, params.N), np.uint32)
    _lib().orc_cmux_tree_read(_p(params), pa, pt, int(v), ctypes.c_void_p(out.ctypes.data))
    return out


def ram_write(params, addr_trgsw, v, new_cell, cells):
    a, pa = _c(addr_trgsw, np.uint32)
    nc, pn = _c(new_cell, np.uint32)
    cells = np.array(cells, np.uint32, copy=True, order="C")
    _lib().orc_ram_write(_p(params), pa, int(v), pn, ctypes.c_void_p(cells.ctypes.data))
    return cells


def extprod_count() -> int:
    return int(_lib().orc_extprod_count())


def extprod_count_reset() -> None:
    _lib().orc_extprod_count_reset()


def ram_cycle(params, bsk, ksk, addr_trgsw, v, flag, wdata, cells):
    """One RAM cycle (reading R14): returns (read data u32[w][n+1], new cells
    u32[w][2^v][2][N]); cells is not modified."""
    bsk, pb = _c(bsk, np.uint32)
    ksk, pk = _c(ksk, np.uint32)
    a, pa = _c(addr_trgsw, np.uint32)
    f, pf = _c(flag, np.uint32)
    wd, pw = _c(wdata, np.uint32)
    new = np.array(cells, dtype=np.uint32, copy=True, order="C")
    w = wd.shape[0]
    rd = np.zeros((w, params.n + 1), np.uint32)
    _lib().orc_ram_cycle(_p(params), pb, pk, pa, v, w, pf, pw, ctypes.c_void_p(new.ctypes.data),
                         ctypes.c_void_p(rd.ctypes.data))
    return rd, new


def rom_read(params, ksk, addr_trgsw, table, v, w):
    """ROM read with vertical and horizontal packing (reading R15): returns (TRLWE
    u32[2][N] holding the word at coefficients 0..w-1, TLWE lvl0 bits u32[w][n+1])."""
    ksk, pk = _c(ksk, np.uint32)
    a, pa = _c(addr_trgsw, np.uint32)
    t, pt = _c(table, np.uint32)
    trlwe = np.zeros((2, params.N), np.uint32)
    bits = np.zeros((w, params.n + 1), np.uint32)
    _lib().orc_rom_read(_p(params), pk, pa, pt, v, w, ctypes.c_void_p(trlwe.ctypes.data),
                        ctypes.c_void_p(bits.ctypes.data))
    return trlwe, bits


# ---- circuit bootstrapping (reading R16): Torus64 primitives and the CB steps ----------

def _out(shape, dtype):
    o = np.zeros(shape, dtype)
    return o, ctypes.c_void_p(o.ctypes.data)


def poly_mul64(a_int, b_torus):
    a, pa = _c(a_int, np.int32)
    b, pb = _c(b_torus, np.uint64)
    o, po = _out(a.size, np.uint64)
    _lib().orc64_poly_mul(a.size, pa, pb, po)
    return o


def rotate64(p, k):
    a, pa = _c(p, np.uint64)
    o, po = _out(a.size, np.uint64)
    _lib().orc64_rotate(a.size, int(k), pa, po)
    return o


def decompose64(l, Bgbit, t):
    o, po = _out(l, np.int32)
    _lib().orc64_decompose(l, Bgbit, int(t) & (2**64 - 1), po)
    return o


def tlwe2_phase(s2, c):
    s, ps = _c(s2, np.uint32)
    c, pc = _c(c, np.uint64)
    return int(_lib().orc64_tlwe_phase(s.size, ps, pc))


def trlwe2_phase(s2, c):
    s, ps = _c(s2, np.uint32)
    c, pc = _c(c, np.uint64)
    o, po = _out(s.size, np.uint64)
    _lib().orc64_trlwe_phase(s.size, ps, pc, po)
    return o


def external_product64(l, Bgbit, C, d):
    C, pC = _c(C, np.uint64)
    d, pd = _c(d, np.uint64)
    o, po = _out(d.shape, np.uint64)
    _lib().orc64_external_product(d.shape[-1], l, Bgbit, pC, pd, po)
    return o


def cmux64(l, Bgbit, C, d1, d0):
    C, pC = _c(C, np.uint64)
    d1, p1 = _c(d1, np.uint64)
    d0, p0 = _c(d0, np.uint64)
    o, po = _out(d0.shape, np.uint64)
    _lib().orc64_cmux(d0.shape[-1], l, Bgbit, pC, p1, p0, po)
    return o


def blind_rotate64(params, cbp, bsk2, bar, mu):
    b, pb = _c(bsk2, np.uint64)
    bar, pbar = _c(bar, np.uint32)
    o, po = _out((2, cbp.N2), np.uint64)
    _lib().orc64_blind_rotate(_p(params), _q(cbp), pb, pbar, int(mu) & (2**64 - 1), po)
    return o


def sample_extract64(trlwe):
    c, pc = _c(trlwe, np.uint64)
    N = c.shape[-1]
    o, po = _out(N + 1, np.uint64)
    _lib().orc64_sample_extract(N, pc, po)
    return o


def cb_tlwe2(params, cbp, bsk2, tlwe0, u):
    """Step 1 of circuit bootstrapping for level u (1..l): lvl2 TLWE u64[N2+1] of m/Bg^u."""
    b, pb = _c(bsk2, np.uint64)
    c, pc = _c(tlwe0, np.uint32)
    o, po = _out(cbp.N2 + 1, np.uint64)
    _lib().orc_cb_tlwe2(_p(params), _q(cbp), pb, pc, int(u), po)
    return o


def pks_digits(t, basebit, a):
    o, po = _out(t, np.uint32)
    _lib().orc_pks_digits(t, basebit, int(a) & (2**64 - 1), po)
    return o


def private_keyswitch(params, cbp, pksk, z, tlwe2):
    """Private functional key switch of a lvl2 TLWE to a lvl1 TRLWE u32[2][N]
    (z = 0: f(x) = -s1[X] x, z = 1: f(x) = x)."""
    k, pk = _c(pksk, np.uint32)
    c, pc = _c(tlwe2, np.uint64)
    o, po = _out((2, params.N), np.uint32)
    _lib().orc_private_keyswitch(_p(params), _q(cbp), pk, int(z), pc, po)
    return o


def circuit_bootstrap(params, cbp, bsk2, pksk, tlwe0, threads: int | None = None):
    """Circuit bootstrapping of one lvl0 TLWE (u32[n+1]) or a batch (u32[R][n+1]) to
    TRGSW lvl1 u32[(R)][2l][2][N]; one input per thread."""
    b, pb = _c(bsk2, np.uint64)
    k, pk = _c(pksk, np.uint32)
    c = np.ascontiguousarray(tlwe0, np.uint32)
    flat = c.reshape(-1, params.n + 1)
    out = np.zeros((flat.shape[0], 2 * params.l, 2, params.N), np.uint32)
    lib, pp, pq = _lib(), _p(params), _q(cbp)

    def one(r):
        lib.orc_circuit_bootstrap(pp, pq, pb, pk, ctypes.c_void_p(flat[r].ctypes.data),
                                  ctypes.c_void_p(out[r].ctypes.data))

    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max(1, min(threads, flat.shape[0]))) as ex:
        list(ex.map(one, range(flat.shape[0])))
    return out if c.ndim > 1 else out[0]
