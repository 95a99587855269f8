"""Python binding of the B300 TFHE gate-bootstrapping library (libtfhe_b300.so).

Argument marshalling only: every step of the evaluated path runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (uint32 for ciphertexts, uint8
gate types, int32 indices); the stream is torch's current CUDA stream unless given.

The raw C entry points are available under their C names (``tfhe_gate_batch`` ...)
on ``lib()``; ``Context`` wraps them.  There is no CPU fallback: if the shared
library is missing or cannot be loaded, importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import functools
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# TFHE_B300_BOUNDS=1 selects the debug build with device index checks (TFHE_EBOUNDS)
LIB_PATH = os.path.join(_HERE, "libtfhe_b300_bounds.so" if os.environ.get("TFHE_B300_BOUNDS") == "1"
                        else "libtfhe_b300.so")

TFHE_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EUNSUPPORTED",
          -6: "ENOKEYS", -7: "EBOUNDS"}
FORM_NTT = 0
FORM_TC = 1
FORM_NTT2 = 2
FORM_AUTO = -1
TC_SINGLE_SM = 0
TC_SM_PAIR = 1
GATES = ["NAND", "AND", "OR", "NOR", "XOR", "XNOR", "ANDNY", "ANDYN", "ORNY", "ORYN"]

# every symbol the public header declares
EXPORTS = [
    "tfhe_version", "tfhe_ctx_create", "tfhe_ctx_destroy", "tfhe_last_error",
    "tfhe_last_error_string",
    "tfhe_ctx_set_keys", "tfhe_ctx_reserve", "tfhe_ctx_sync", "tfhe_gate_batch",
    "tfhe_gate_batch_host", "tfhe_blind_rotate", "tfhe_extract_keyswitch", "tfhe_cmux_batch",
    "tfhe_cmux_tree_read", "tfhe_ram_write", "tfhe_circuit_plan", "tfhe_plan_num_levels",
    "tfhe_plan_circuit_last_level", "tfhe_plan_run", "tfhe_plan_run_dataflow", "tfhe_plan_destroy",
    "tfhe_ctx_enable_timing", "tfhe_ctx_stage_times", "tfhe_gate_batch_noalloc",
    "tfhe_ctx_set_tc_level",
    "tfhe_ctx_tc_level",
    "tfhe_ctx_set_tc_variant",
    "tfhe_ctx_tc_variant",
    "tfhe_ctx_set_tc_pass_limit",
    "tfhe_ctx_autotune",
    "tfhe_ctx_tune_table",
    "tfhe_mux_batch",
    "tfhe_mux_batch_noks",
    "tfhe_ram_cycle",
    "tfhe_rom_read",
    "tfhe_ctx_set_cb_keys",
    "tfhe_circuit_bootstrap",
    "tfhe_cb_tlwe2",
    "tfhe_private_keyswitch",
    "tfhe_ctx_probe_wait",
]
STAGES = ["combine", "blind_rotate_ntt", "tc_aux", "blind_rotate_tc", "keyswitch", "cmux",
          "cb_blind_rotate", "cb_keyswitch"]
NUM_STAGES = 8


class TfheError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class CParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("N", ctypes.c_int32), ("l", ctypes.c_int32),
                ("Bgbit", ctypes.c_int32), ("ks_t", ctypes.c_int32),
                ("ks_basebit", ctypes.c_int32)]


class CCbParams(ctypes.Structure):
    _fields_ = [("N2", ctypes.c_int32), ("l2", ctypes.c_int32), ("Bg2bit", ctypes.c_int32),
                ("pks_t", ctypes.c_int32), ("pks_basebit", ctypes.c_int32)]


class CCircuit(ctypes.Structure):
    _fields_ = [("num_inputs", ctypes.c_int32), ("num_gates", ctypes.c_int32),
                ("types", ctypes.c_void_p), ("in_idx", ctypes.c_void_p)]


@functools.lru_cache(maxsize=1)
def lib():
    """Load the in-tree shared library (raises if it has not been built)."""
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2010_09410_b300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "tfhe_version": (i32, []),
        "tfhe_ctx_create": (i32, [ctypes.POINTER(CParams), i32, ctypes.POINTER(vp)]),
        "tfhe_ctx_destroy": (None, [vp]),
        "tfhe_last_error": (ctypes.c_char_p, [vp]),
        "tfhe_last_error_string": (i32, [vp, ctypes.c_char_p, i32]),
        "tfhe_ctx_set_keys": (i32, [vp, vp, vp, vp]),
        "tfhe_ctx_reserve": (i32, [vp, i32]),
        "tfhe_ctx_sync": (i32, [vp, vp]),
        "tfhe_gate_batch": (i32, [vp, vp, i64, vp, vp, vp, i32, i32, vp]),
        "tfhe_gate_batch_host": (i32, [vp, vp, i64, vp, vp, vp, i32, i32, vp]),
        "tfhe_blind_rotate": (i32, [vp, vp, vp, i32, i32, vp]),
        "tfhe_extract_keyswitch": (i32, [vp, vp, vp, i32, vp]),
        "tfhe_cmux_batch": (i32, [vp, vp, i32, vp, vp, vp, i32, i32, vp]),
        "tfhe_cmux_tree_read": (i32, [vp, vp, vp, i32, vp, i32, i32, vp]),
        "tfhe_ram_write": (i32, [vp, vp, i32, vp, vp, i32, vp]),
        "tfhe_circuit_plan": (i32, [vp, ctypes.POINTER(CCircuit), i32, i32, ctypes.POINTER(vp)]),
        "tfhe_plan_num_levels": (i32, [vp]),
        "tfhe_plan_circuit_last_level": (i32, [vp, i32]),
        "tfhe_plan_run": (i32, [vp, vp, vp, i32, vp, vp]),
        "tfhe_plan_run_dataflow": (i32, [vp, vp, vp, vp]),
        "tfhe_plan_destroy": (None, [vp]),
        "tfhe_ctx_enable_timing": (i32, [vp, i32]),
        "tfhe_ctx_stage_times": (i32, [vp, vp, vp]),
        "tfhe_gate_batch_noalloc": (i32, [vp, vp, i64, vp, vp, vp, i32, vp]),
        "tfhe_ctx_set_tc_level": (i32, [vp, i32]),
        "tfhe_ctx_tc_level": (i32, [vp]),
        "tfhe_ctx_set_tc_variant": (i32, [vp, i32]),
        "tfhe_ctx_tc_variant": (i32, [vp]),
        "tfhe_ctx_set_tc_pass_limit": (i32, [vp, i32]),
        "tfhe_ctx_autotune": (i32, [vp, i32, vp]),
        "tfhe_ctx_tune_table": (i32, [vp, vp, vp, vp, vp, i32]),
        "tfhe_mux_batch": (i32, [vp, vp, i64, vp, vp, i32, i32, vp]),
        "tfhe_mux_batch_noks": (i32, [vp, vp, i64, vp, vp, i32, i32, vp]),
        "tfhe_ram_cycle": (i32, [vp, vp, i32, i32, vp, vp, vp, vp, i32, vp]),
        "tfhe_rom_read": (i32, [vp, vp, vp, i32, i32, vp, vp, i32, vp]),
        "tfhe_ctx_set_cb_keys": (i32, [vp, ctypes.POINTER(CCbParams), vp, vp, vp]),
        "tfhe_circuit_bootstrap": (i32, [vp, vp, vp, i32, vp]),
        "tfhe_cb_tlwe2": (i32, [vp, vp, vp, i32, vp]),
        "tfhe_private_keyswitch": (i32, [vp, vp, vp, i32, i32, vp]),
        "tfhe_ctx_probe_wait": (i32, [vp, vp, ctypes.c_uint32, i64, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _ptr(t):
    """Device (or host) address of a torch tensor or numpy array, None passes NULL."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A library context on one CUDA device: parameters, keys and workspaces."""

    def __init__(self, params, device: int = 0):
        p = params.abi() if hasattr(params, "abi") else tuple(params)
        self.params = params
        self.n, self.N, self.l = p[0], p[1], p[2]
        self.device = device
        h = ctypes.c_void_p()
        rc = lib().tfhe_ctx_create(ctypes.byref(CParams(*p)), device, ctypes.byref(h))
        if rc != TFHE_OK:
            raise TfheError(rc, "tfhe_ctx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().tfhe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != TFHE_OK:
            raise TfheError(rc, f"{what}: {lib().tfhe_last_error(self.h).decode()}")

    def set_keys(self, bsk, ksk, stream=None):
        self._check(lib().tfhe_ctx_set_keys(self.h, _ptr(bsk), _ptr(ksk), _stream(stream)),
                    "set_keys")

    def set_tc_level(self, levels: int):
        """Karatsuba levels of the tensor-core form (0, 1, 2; -1 = default)."""
        self._check(lib().tfhe_ctx_set_tc_level(self.h, levels), "set_tc_level")

    def tc_level(self) -> int:
        """Karatsuba level the tensor-core form runs with."""
        rc = lib().tfhe_ctx_tc_level(self.h)
        self._check(min(rc, 0), "tc_level")
        return rc

    def set_tc_variant(self, variant: int):
        """TC_SINGLE_SM, TC_SM_PAIR or -1 (default) for the tensor-core BlindRotate."""
        self._check(lib().tfhe_ctx_set_tc_variant(self.h, variant), "set_tc_variant")

    def tc_variant(self) -> int:
        rc = lib().tfhe_ctx_tc_variant(self.h)
        self._check(min(rc, 0), "tc_variant")
        return rc

    def set_tc_pass_limit(self, limit: int):
        """Largest per-gate sum of |digit| accumulated in one TMEM pass (0 .. 2^17, -1 default)."""
        self._check(lib().tfhe_ctx_set_tc_pass_limit(self.h, limit), "set_tc_pass_limit")

    def autotune(self, max_gates: int, stream=None):
        """Time every form / Karatsuba level per batch width; plans with form -1 use it."""
        self._check(lib().tfhe_ctx_autotune(self.h, max_gates, _stream(stream)), "autotune")
        return self.tune_table()

    def tune_table(self):
        """[(width, form, tc_level, ms)] measured by autotune (empty before)."""
        n = lib().tfhe_ctx_tune_table(self.h, None, None, None, None, 0)
        w, f, lv = (ctypes.c_int * max(n, 1))(), (ctypes.c_int * max(n, 1))(), (ctypes.c_int * max(n, 1))()
        ms = (ctypes.c_float * max(n, 1))()
        lib().tfhe_ctx_tune_table(self.h, w, f, lv, ms, n)
        return [(w[i], f[i], lv[i], ms[i]) for i in range(n)]

    def enable_timing(self, on: bool = True):
        self._check(lib().tfhe_ctx_enable_timing(self.h, 1 if on else 0), "enable_timing")

    def stage_times(self):
        """{stage: (total ms, launches)} since the last call; waits for the events."""
        ms = (ctypes.c_double * NUM_STAGES)()
        n = (ctypes.c_int64 * NUM_STAGES)()
        self._check(lib().tfhe_ctx_stage_times(self.h, ms, n), "stage_times")
        return {name: (ms[i], n[i]) for i, name in enumerate(STAGES)}

    def reserve(self, max_gates: int):
        self._check(lib().tfhe_ctx_reserve(self.h, max_gates), "reserve")

    def probe_wait(self, flag, target: int, max_cycles: int, stream=None):
        """One bounded device wait on flag (device u32) >= target; a time-out shows up as
        TFHE_ETIMEOUT at the next sync."""
        self._check(lib().tfhe_ctx_probe_wait(self.h, _ptr(flag), target, max_cycles,
                                              _stream(stream)), "probe_wait")

    def sync(self, stream=None):
        self._check(lib().tfhe_ctx_sync(self.h, _stream(stream)), "sync")

    def gate_batch(self, inp, types, idx, out, form=FORM_NTT, stream=None):
        G = types.numel()
        self._check(lib().tfhe_gate_batch(self.h, _ptr(inp), inp.shape[0], _ptr(types),
                                          _ptr(idx), _ptr(out), G, form, _stream(stream)),
                    "gate_batch")
        return out

    def mux_batch(self, inp, idx3, out, form=FORM_NTT, stream=None, noks=False):
        """HomMUX of rows idx3[g] = (selector, taken if 1, taken if 0); TLWE out [G][n+1],
        or with noks the TRLWE before SampleExtract and key switching [G][2][N]."""
        fn = lib().tfhe_mux_batch_noks if noks else lib().tfhe_mux_batch
        self._check(fn(self.h, _ptr(inp), inp.shape[0], _ptr(idx3), _ptr(out), idx3.shape[0],
                       form, _stream(stream)), "mux_batch")
        return out

    def gate_batch_noalloc(self, inp, types, idx, out, stream=None):
        """tfhe_gate_batch_noalloc: NTT form, scratch in the library's fixed device array."""
        self._check(lib().tfhe_gate_batch_noalloc(self.h, _ptr(inp), inp.shape[0], _ptr(types),
                                                  _ptr(idx), _ptr(out), types.numel(),
                                                  _stream(stream)), "gate_batch_noalloc")
        return out

    def gate_batch_host(self, inp, types, idx, out, form=FORM_NTT, stream=None):
        """Host (numpy or CPU torch) buffers in and out; returns when `out` is filled."""
        G = types.size if hasattr(types, "size") and not callable(types.size) else types.numel()
        self._check(lib().tfhe_gate_batch_host(self.h, _ptr(inp), inp.shape[0], _ptr(types),
                                               _ptr(idx), _ptr(out), G, form, _stream(stream)),
                    "gate_batch_host")
        return out

    def blind_rotate(self, bar, acc, form=FORM_NTT, stream=None):
        self._check(lib().tfhe_blind_rotate(self.h, _ptr(bar), _ptr(acc), bar.shape[0], form,
                                            _stream(stream)), "blind_rotate")
        return acc

    def extract_keyswitch(self, acc, out, stream=None):
        self._check(lib().tfhe_extract_keyswitch(self.h, _ptr(acc), _ptr(out), acc.shape[0],
                                                 _stream(stream)), "extract_keyswitch")
        return out

    def cmux_batch(self, trgsw, group, d1, d0, out, form=FORM_NTT, stream=None):
        self._check(lib().tfhe_cmux_batch(self.h, _ptr(trgsw), group, _ptr(d1), _ptr(d0),
                                          _ptr(out), d1.shape[0], form, _stream(stream)),
                    "cmux_batch")
        return out

    def cmux_tree_read(self, addr_trgsw, table, v, out, form=FORM_NTT, stream=None):
        self._check(lib().tfhe_cmux_tree_read(self.h, _ptr(addr_trgsw), _ptr(table), v, _ptr(out),
                                              out.shape[0], form, _stream(stream)),
                    "cmux_tree_read")
        return out

    def ram_write(self, addr_trgsw, v, new_cell, cells, form=FORM_NTT, stream=None):
        self._check(lib().tfhe_ram_write(self.h, _ptr(addr_trgsw), v, _ptr(new_cell), _ptr(cells),
                                         form, _stream(stream)), "ram_write")
        return cells

    def ram_cycle(self, addr_trgsw, v, flag, wdata, cells, rdata, form=FORM_TC, stream=None):
        """One RAM cycle: reads rdata [w][n+1] at the address, writes if flag, refreshes."""
        self._check(lib().tfhe_ram_cycle(self.h, _ptr(addr_trgsw), v, wdata.shape[0], _ptr(flag),
                                         _ptr(wdata), _ptr(cells), _ptr(rdata), form,
                                         _stream(stream)), "ram_cycle")
        return rdata

    def rom_read(self, addr_trgsw, table, v, w, out_trlwe=None, out_bits=None, stream=None):
        """Packed ROM read: out_trlwe [R][2][N] and/or out_bits [R][w][n+1]."""
        R = addr_trgsw.shape[0]
        self._check(lib().tfhe_rom_read(self.h, _ptr(addr_trgsw), _ptr(table), v, w,
                                        _ptr(out_trlwe) if out_trlwe is not None else None,
                                        _ptr(out_bits) if out_bits is not None else None, R,
                                        _stream(stream)), "rom_read")
        return out_trlwe, out_bits

    def set_cb_keys(self, cbp, bsk2, pksk, stream=None):
        """Circuit-bootstrapping keys: BSK2 u64[n][2 l2][2][N2] (a torch int64/uint64 tensor)
        and PKSK u32[2][N2+1][t][2^basebit][2][N]."""
        q = cbp.abi() if hasattr(cbp, "abi") else tuple(cbp)
        self._check(lib().tfhe_ctx_set_cb_keys(self.h, ctypes.byref(CCbParams(*q)), _ptr(bsk2),
                                               _ptr(pksk), _stream(stream)), "set_cb_keys")

    def circuit_bootstrap(self, tlwe, out, stream=None):
        """lvl0 TLWE [R][n+1] -> lvl1 TRGSW [R][2l][2][N]."""
        self._check(lib().tfhe_circuit_bootstrap(self.h, _ptr(tlwe), _ptr(out), tlwe.shape[0],
                                                 _stream(stream)), "circuit_bootstrap")
        return out

    def cb_tlwe2(self, tlwe, out, stream=None):
        """Step 1 of circuit bootstrapping: lvl0 TLWE [R][n+1] -> lvl2 TLWE [R][l][N2+1]."""
        self._check(lib().tfhe_cb_tlwe2(self.h, _ptr(tlwe), _ptr(out), tlwe.shape[0],
                                        _stream(stream)), "cb_tlwe2")
        return out

    def private_keyswitch(self, tlwe2, out, z, stream=None):
        """Step 2: lvl2 TLWE [J][N2+1] -> TRLWE [J][2][N] with f_0 = -s1[X] x or f_1 = x."""
        self._check(lib().tfhe_private_keyswitch(self.h, _ptr(tlwe2), _ptr(out), tlwe2.shape[0],
                                                 z, _stream(stream)), "private_keyswitch")
        return out

    def plan(self, circuits, form=FORM_AUTO):
        return Plan(self, circuits, form)


class Plan:
    """A level schedule for one or more circuits (host numpy wiring)."""

    def __init__(self, ctx: Context, circuits, form=FORM_AUTO):
        import numpy as np
        self.ctx = ctx
        self._keep = []
        arr = (CCircuit * len(circuits))()
        for i, c in enumerate(circuits):
            t = np.ascontiguousarray(c.types, np.uint8)
            x = np.ascontiguousarray(c.idx, np.int32)
            self._keep += [t, x]
            arr[i] = CCircuit(c.num_inputs, t.size, t.ctypes.data, x.ctypes.data)
        h = ctypes.c_void_p()
        ctx._check(lib().tfhe_circuit_plan(ctx.h, arr, len(circuits), form, ctypes.byref(h)),
                   "circuit_plan")
        self.h = h
        self.num_levels = lib().tfhe_plan_num_levels(h)
        self.circuit_last_level = [lib().tfhe_plan_circuit_last_level(h, i)
                                   for i in range(len(circuits))]

    def run(self, primary_in, gate_out, use_graph=False, level_events=None, stream=None):
        ev = None
        if level_events is not None:
            for e in level_events:
                if not e.cuda_event:  # torch creates the CUDA event at its first record
                    e.record()
            ev = (ctypes.c_void_p * len(level_events))(*[e.cuda_event for e in level_events])
        self.ctx._check(lib().tfhe_plan_run(self.h, _ptr(primary_in), _ptr(gate_out),
                                            1 if use_graph else 0, ev, _stream(stream)),
                        "plan_run")
        return gate_out

    def run_dataflow(self, primary_in, gate_out, stream=None):
        """All gates in the two-prime per-gate form, each started once its inputs exist."""
        self.ctx._check(lib().tfhe_plan_run_dataflow(self.h, _ptr(primary_in), _ptr(gate_out),
                                                     _stream(stream)), "plan_run_dataflow")
        return gate_out

    def close(self):
        if getattr(self, "h", None):
            lib().tfhe_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
