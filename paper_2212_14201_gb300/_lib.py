"""ctypes binding of libqsim: one Python function per C entry point, same names.

Argument marshalling only -- every step of the simulation runs in the library's
CUDA kernels.  Importing this module does not load the library; the first call
does, and raises QsimError if libqsim.so has not been built (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsim.so")

QS_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "UNSUPPORTED"}

PLAN_PLAIN, PLAN_GREEDY, PLAN_LEARNED = 0, 1, 2

GATE_DTYPE = np.dtype([
    ("type", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("param_idx", "<i4"),
    ("ctrl_mask", "<u8"), ("p", "<f8", (3,)), ("dagger", "<i4"), ("reserved", "<i4"),
], align=True)
PAULI_DTYPE = np.dtype([("coef", "<f8"), ("xmask", "<u8"), ("zmask", "<u8")], align=True)
NOISE_DTYPE = np.dtype([("model", "<i4"), ("gate_type", "<i4"), ("q0", "<i4"), ("q1", "<i4"),
                        ("p", "<f8"), ("t1", "<f8"), ("t2", "<f8"), ("tgate", "<f8")], align=True)
PINSTR_DTYPE = np.dtype([
    ("op", "<i4"), ("qubit", "<i4"), ("dst", "<i4"), ("alu", "<i4"), ("lhs", "<i4"), ("rhs", "<i4"),
    ("imm", "<i8"), ("n_then", "<u4"), ("n_else", "<u4"), ("gate_begin", "<u8"), ("gate_end", "<u8"),
], align=True)


class QsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libqsim {ERRORS.get(code, code)}: {msg}")
        self.code = code


class PlanStats(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_int64), ("n_passes", ctypes.c_int64), ("n_tile_passes", ctypes.c_int64),
                ("n_dense", ctypes.c_int64), ("est_seconds", ctypes.c_double), ("tile_qubits", ctypes.c_int64),
                ("learned_fallback", ctypes.c_int64)]


class PassOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("target", ctypes.c_int32), ("ctrl_mask", ctypes.c_uint64),
                ("m", ctypes.c_double * 8), ("table", ctypes.c_int32), ("bits", ctypes.c_int32),
                ("nsigns", ctypes.c_int32), ("sign_q", ctypes.c_uint8 * 16), ("sign_t", ctypes.c_uint8 * 16)]


class TimingRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("k", ctypes.c_int32), ("n_ops", ctypes.c_int32),
                ("qubit_mask", ctypes.c_uint64), ("ctrl_mask", ctypes.c_uint64), ("items", ctypes.c_double),
                ("flops", ctypes.c_double), ("int_ops", ctypes.c_double), ("ms", ctypes.c_double)]


K_PHASE1, K_DIAG, K_ANTI, K_REAL, K_GENERAL, K_DENSE, K_TILE, K_REDUCE, K_ADJOINT, K_OTHER = 1, 2, 3, 4, 5, 10, 11, 20, 30, 40

_lock = threading.Lock()
_lib = None

P, I32, U64, SZ, DBL = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)

SIGNATURES = {
    "qs_last_error": (ctypes.c_char_p, []),
    "qs_max_qubits": (I32, []),
    "qs_fault_set": (I32, [I32, ctypes.c_longlong, ctypes.c_longlong]),
    "qs_fault_get": (I32, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                           ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                           ctypes.POINTER(ctypes.c_int)]),
    "qs_alloc": (I32, [I32, P, PP]),
    "qs_alloc_external": (I32, [I32, P, P, PP]),
    "qs_alloc_c64": (I32, [I32, P, PP]),
    "qs_state_precision": (I32, [P, ctypes.POINTER(ctypes.c_int)]),
    "qs_free": (I32, [P]),
    "qs_num_qubits": (I32, [P]),
    "qs_device_ptr": (I32, [P, PP]),
    "qs_set_zero": (I32, [P]),
    "qs_set_state": (I32, [P, P, I32]),
    "qs_get_state": (I32, [P, P, I32]),
    "qs_sync": (I32, [P]),
    "qs_set_arith": (I32, [P, I32]),
    "qs_state_modified": (I32, [P]),
    "qs_apply": (I32, [P, P, SZ, P, P]),
    "qs_apply_matrix": (I32, [P, P, I32, U64, P]),
    "qs_gate_list_dagger": (I32, [P, SZ, P]),
    "qs_plan_create": (I32, [I32, P, SZ, I32, I32, PP]),
    "qs_plan_free": (I32, [P]),
    "qs_plan_create_tiled": (I32, [I32, P, SZ, I32, PP]),
    "qs_plan_create_variant": (I32, [I32, P, SZ, I32, I32, PP]),
    "qs_plan_get_stats": (I32, [P, ctypes.POINTER(PlanStats)]),
    "qs_plan_pass_info": (I32, [P, SZ, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint64), P, SZ,
                                ctypes.POINTER(SZ)]),
    "qs_probs": (I32, [P, P, I32, P, I32]),
    "qs_probs_dict": (I32, [P, P, I32, DBL, P, P, SZ, ctypes.POINTER(SZ)]),
    "qs_expect_z_all": (I32, [P, P]),
    "qs_expect_pauli": (I32, [P, P, SZ, ctypes.POINTER(DBL)]),
    "qs_sample": (I32, [P, U64, U64, P, I32]),
    "qs_adjoint_grad": (I32, [P, P, SZ, P, SZ, P, SZ, ctypes.POINTER(DBL), P]),
    "qs_expect_z_all_noalloc": (I32, [P, I32, P, P]),
    "qs_set_adjoint_fused": (I32, [I32]),
    "qs_set_aggregate": (I32, [I32]),
    "qs_set_phase_tables": (I32, [I32]),
    "qs_set_rotation_pairs": (I32, [I32]),
    "qs_plan_pass_ops": (I32, [P, SZ, P, SZ, P, I32, ctypes.POINTER(PassOp), SZ, ctypes.POINTER(SZ), P, SZ,
                               ctypes.POINTER(SZ)]),
    "qs_mlp_create": (I32, [I32, I32, P, U64, PP]),
    "qs_mlp_free": (I32, [P]),
    "qs_mlp_num_weights": (I32, [P, ctypes.POINTER(SZ)]),
    "qs_mlp_get_weights": (I32, [P, P]),
    "qs_mlp_set_weights": (I32, [P, P]),
    "qs_mlp_forward": (I32, [P, P, SZ, P]),
    "qs_mlp_loss_grad": (I32, [P, P, P, SZ, ctypes.POINTER(DBL), P]),
    "qs_mlp_train": (I32, [P, P, P, SZ, I32, DBL, ctypes.POINTER(DBL)]),
    "qs_plan_features": (I32, [P, P, SZ, P]),
    "qs_plan_create_learned": (I32, [I32, P, SZ, P, PP]),
    "qs_plan_create_scored": (I32, [I32, P, SZ, P, P, PP]),
    "qs_plan_pass_kernel_ops": (I32, [P, SZ, P, SZ, P, P, ctypes.POINTER(DBL)]),
    "qs_batch_create": (I32, [SZ, P, P, P, P, P, P, PP]),
    "qs_batch_run": (I32, [P, P, P, P, I32]),
    "qs_batch_last_ms": (I32, [P, ctypes.POINTER(DBL)]),
    "qs_batch_info": (I32, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(SZ)]),
    "qs_batch_cluster": (I32, [P, ctypes.POINTER(ctypes.c_int)]),
    "qs_measure": (I32, [P, I32, DBL, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(DBL)]),
    "qs_run_noisy": (I32, [P, P, SZ, P, P, SZ, DBL, U64, I32, ctypes.POINTER(U64)]),
    "qs_readout_error": (I32, [P, SZ, I32, DBL, DBL, U64, I32, P]),
    "qs_partial_amplitudes": (I32, [I32, P, SZ, P, I32, P, SZ, P, I32, P, ctypes.POINTER(U64)]),
    "qs_run_program": (I32, [P, P, SZ, P, SZ, P, I32, U64, U64, P, SZ, P, SZ, ctypes.POINTER(U64)]),
    "qs_set_batch_cluster": (I32, [I32]),
    "qs_batch_free": (I32, [P]),
    "qs_timing_enable": (I32, [P, I32]),
    "qs_timing_fetch": (I32, [P, ctypes.POINTER(TimingRecord), SZ, ctypes.POINTER(SZ)]),
    "qs_launch_count": (U64, []),
}


def lib():
    """The loaded library (raises QsimError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise QsimError(-3, f"{LIB_PATH} is missing: build it with paper_2212_14201_gb300.build()")
            l = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


def _chk(rc: int):
    if rc != QS_OK:
        raise QsimError(rc, lib().qs_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _host_or_dev(x):
    """(pointer, on_device) of a numpy array or a CUDA torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (1 if x.is_cuda else 0)
    raise TypeError(f"expected numpy array or torch tensor, got {type(x)}")


def as_gates(gates) -> np.ndarray:
    g = np.ascontiguousarray(gates)
    if g.dtype != GATE_DTYPE:
        g = g.astype(GATE_DTYPE)
    return g


def as_paulis(terms) -> np.ndarray:
    t = np.ascontiguousarray(terms)
    if t.dtype != PAULI_DTYPE:
        t = t.astype(PAULI_DTYPE)
    return t


# ---- one wrapper per entry point ---------------------------------------------------

def qs_last_error() -> str:
    return lib().qs_last_error().decode()


def qs_max_qubits() -> int:
    return lib().qs_max_qubits()


FAULT_NONE, FAULT_ALLOC, FAULT_LAUNCH = 0, 1, 2


def qs_fault_set(kind: int, after: int = 0, count: int = 1) -> None:
    """Arm the host-side fault: the first `after` events of `kind` pass, the next
    `count` fail (-1: all); FAULT_NONE disarms."""
    _chk(lib().qs_fault_set(kind, after, count))


def qs_fault_get() -> dict:
    k, env = ctypes.c_int(), ctypes.c_int()
    a, l, f = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _chk(lib().qs_fault_get(ctypes.byref(k), ctypes.byref(a), ctypes.byref(l), ctypes.byref(f), ctypes.byref(env)))
    return {"kind": k.value, "after": a.value, "left": l.value, "fired": f.value, "env_status": env.value}


def qs_alloc(n: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _chk(lib().qs_alloc(n, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def qs_alloc_external(n: int, device_amps, stream=None) -> int:
    ptr = device_amps if isinstance(device_amps, int) else device_amps.data_ptr()
    h = ctypes.c_void_p()
    _chk(lib().qs_alloc_external(n, ptr, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def qs_free(h: int):
    _chk(lib().qs_free(h))


def qs_num_qubits(h: int) -> int:
    r = lib().qs_num_qubits(h)
    if r < 0:
        _chk(r)
    return r


def qs_device_ptr(h: int) -> int:
    p = ctypes.c_void_p()
    _chk(lib().qs_device_ptr(h, ctypes.byref(p)))
    return p.value


def qs_set_zero(h: int):
    _chk(lib().qs_set_zero(h))


def qs_alloc_c64(n: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _chk(lib().qs_alloc_c64(n, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def qs_state_precision(h: int) -> int:
    b = ctypes.c_int()
    _chk(lib().qs_state_precision(h, ctypes.byref(b)))
    return b.value


def _check_amps(h: int, x):
    """The buffer's element size must match the state's precision and length."""
    n = qs_num_qubits(h)
    bits = qs_state_precision(h)
    item = x.itemsize if isinstance(x, np.ndarray) else x.element_size()
    numel = x.size if isinstance(x, np.ndarray) else x.numel()
    comp = 8 if bits == 128 else 4            # bytes per real component
    if item not in (comp, 2 * comp) or numel * item != (2 << n) * comp:
        raise ValueError(f"buffer does not hold 2^{n} complex{bits} amplitudes")


def qs_set_state(h: int, amps):
    _check_amps(h, amps)
    ptr, dev = _host_or_dev(amps)
    _chk(lib().qs_set_state(h, ptr, dev))


def qs_get_state(h: int, out=None):
    """Copy the amplitudes into `out` (numpy array or device tensor of the state's
    precision); with out=None returns a new numpy complex128 (or complex64) array."""
    if out is None:
        n = qs_num_qubits(h)
        out = np.empty(1 << n, dtype=np.complex64 if qs_state_precision(h) == 64 else np.complex128)
    _check_amps(h, out)
    ptr, dev = _host_or_dev(out)
    _chk(lib().qs_get_state(h, ptr, dev))
    return out


def qs_sync(h: int):
    _chk(lib().qs_sync(h))


ARITH_AUTO, ARITH_FP64, ARITH_FIXED = 0, 1, 2


def qs_set_arith(h: int, mode: int):
    _chk(lib().qs_set_arith(h, mode))


def qs_state_modified(h: int):
    _chk(lib().qs_state_modified(h))


def qs_apply(h: int, gates, params=None, plan: int | None = None):
    g = as_gates(gates)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    _chk(lib().qs_apply(h, g.ctypes.data if len(g) else None, len(g),
                        None if pr is None else pr.ctypes.data, plan))


def qs_measure(h: int, qubit: int, u: float):
    """Projective measurement with the draw u: (outcome, p1 / (p0 + p1))."""
    o, p1 = ctypes.c_int(), ctypes.c_double()
    _chk(lib().qs_measure(h, qubit, u, ctypes.byref(o), ctypes.byref(p1)))
    return o.value, p1.value


def qs_run_program(h: int, prog, gates, params=None, fuse: bool = False, seed: int = 0,
                   max_iters: int = 1 << 20, cbits=None, ncbits: int = 8, record_cap: int = 4096):
    """Runs a structured program on the state: returns (cbits, record of p1 per
    measurement)."""
    pg = np.ascontiguousarray(prog)
    if pg.dtype != PINSTR_DTYPE:
        pg = pg.astype(PINSTR_DTYPE)
    g = as_gates(gates)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    cb = np.zeros(ncbits, dtype=np.int64) if cbits is None else np.array(cbits, dtype=np.int64)
    rec = np.zeros(record_cap, dtype=np.float64)
    nm = ctypes.c_uint64()
    _chk(lib().qs_run_program(h, pg.ctypes.data if len(pg) else None, len(pg), g.ctypes.data if len(g) else None,
                              len(g), None if pr is None else pr.ctypes.data, 1 if fuse else 0, seed, max_iters,
                              cb.ctypes.data if len(cb) else None, len(cb), rec.ctypes.data, record_cap,
                              ctypes.byref(nm)))
    return cb, rec[:min(nm.value, record_cap)].copy()


def qs_run_noisy(h: int, gates, rules, params=None, rotation_error: float = 0.0, seed: int = 0,
                 fuse: bool = True) -> int:
    """One noise trajectory on the state; returns the number of draws used."""
    g = as_gates(gates)
    r = np.ascontiguousarray(rules)
    if r.dtype != NOISE_DTYPE:
        r = r.astype(NOISE_DTYPE)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    nd = ctypes.c_uint64()
    _chk(lib().qs_run_noisy(h, g.ctypes.data if len(g) else None, len(g), None if pr is None else pr.ctypes.data,
                            r.ctypes.data if len(r) else None, len(r), rotation_error, seed, 1 if fuse else 0,
                            ctypes.byref(nd)))
    return nd.value


def qs_readout_error(samples, n: int, f0: float, f1: float, seed: int, stream=None):
    """Readout error in place on sampled indices (numpy uint64 array or CUDA tensor)."""
    ptr, dev = _host_or_dev(samples)
    count = samples.size if isinstance(samples, np.ndarray) else samples.numel()
    _chk(lib().qs_readout_error(ptr, count, n, f0, f1, seed, dev, _stream_ptr(stream)))
    return samples


def qs_partial_amplitudes(n: int, gates, n_low: int, indices, params=None, fuse: bool = True, stream=None):
    """Selected amplitudes of an n-qubit program by cutting the gates across the
    split at n_low: (complex128 array, number of paths)."""
    g = as_gates(gates)
    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    out = np.empty(len(idx), dtype=np.complex128)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    npaths = ctypes.c_uint64()
    _chk(lib().qs_partial_amplitudes(n, g.ctypes.data if len(g) else None, len(g),
                                     None if pr is None else pr.ctypes.data, n_low,
                                     idx.ctypes.data if len(idx) else None, len(idx),
                                     out.ctypes.data if len(idx) else None, 1 if fuse else 0,
                                     _stream_ptr(stream), ctypes.byref(npaths)))
    return out, npaths.value


def qs_apply_matrix(h: int, targets, mat, ctrl_mask: int = 0):
    t = np.ascontiguousarray(targets, dtype=np.int32)
    m = np.ascontiguousarray(mat, dtype=np.complex128)
    _chk(lib().qs_apply_matrix(h, t.ctypes.data, len(t), ctrl_mask, m.ctypes.data))


def qs_gate_list_dagger(gates) -> np.ndarray:
    g = as_gates(gates)
    out = np.empty_like(g)
    _chk(lib().qs_gate_list_dagger(g.ctypes.data if len(g) else None, len(g), out.ctypes.data if len(g) else None))
    return out


def qs_plan_create(n: int, gates, mode: int = PLAN_GREEDY, kmax: int = 5) -> int:
    g = as_gates(gates)
    h = ctypes.c_void_p()
    _chk(lib().qs_plan_create(n, g.ctypes.data if len(g) else None, len(g), mode, kmax, ctypes.byref(h)))
    return h.value


def qs_set_adjoint_fused(on: bool):
    _chk(lib().qs_set_adjoint_fused(1 if on else 0))


def qs_set_aggregate(on: bool):
    _chk(lib().qs_set_aggregate(1 if on else 0))


def qs_set_phase_tables(on: bool):
    _chk(lib().qs_set_phase_tables(1 if on else 0))

def qs_set_rotation_pairs(on):
    """Process-wide: run pairs of real rotations as one 4x4 op on quads (Q60 tiles);
    True/1 with phase tables fused into the following pair, 2 without, False/0 off."""
    _chk(lib().qs_set_rotation_pairs(int(on)))


def qs_plan_create_tiled(n: int, gates, tile_qubits: int) -> int:
    g = as_gates(gates)
    h = ctypes.c_void_p()
    _chk(lib().qs_plan_create_tiled(n, g.ctypes.data if len(g) else None, len(g), tile_qubits, ctypes.byref(h)))
    return h.value


def qs_plan_create_variant(n: int, gates, tile_qubits: int, strategy: int) -> int:
    g = as_gates(gates)
    h = ctypes.c_void_p()
    _chk(lib().qs_plan_create_variant(n, g.ctypes.data if len(g) else None, len(g), tile_qubits, strategy,
                                      ctypes.byref(h)))
    return h.value


def qs_plan_free(p: int):
    _chk(lib().qs_plan_free(p))


def qs_plan_get_stats(p: int) -> dict:
    st = PlanStats()
    _chk(lib().qs_plan_get_stats(p, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in PlanStats._fields_}


def qs_plan_pass_info(p: int, i: int):
    """(kind, qubit mask, gate indices) of pass i."""
    kind, qm, cnt = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_size_t()
    _chk(lib().qs_plan_pass_info(p, i, ctypes.byref(kind), ctypes.byref(qm), None, 0, ctypes.byref(cnt)))
    idx = np.empty(max(1, cnt.value), dtype=np.uint32)
    _chk(lib().qs_plan_pass_info(p, i, ctypes.byref(kind), ctypes.byref(qm), idx.ctypes.data, cnt.value,
                                 ctypes.byref(cnt)))
    return kind.value, qm.value, idx[:cnt.value].copy()


def qs_plan_pass_ops(p: int, i: int, gates, params=None, q60: bool = True):
    """(ops, tables) a tile pass runs: ops as dicts (kind 0: target, ctrl_mask,
    2x2 complex matrix; kind 1: table index, bits), tables as an array of
    2^bits complex entries per table (entry j: tile index j)."""
    g = as_gates(gates)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    cnt, nt = ctypes.c_size_t(), ctypes.c_size_t()
    args = (p, i, g.ctypes.data if len(g) else None, len(g), None if pr is None else pr.ctypes.data, 1 if q60 else 0)
    _chk(lib().qs_plan_pass_ops(*args, None, 0, ctypes.byref(cnt), None, 0, ctypes.byref(nt)))
    ops = (PassOp * max(1, cnt.value))()
    _chk(lib().qs_plan_pass_ops(*args, ops, cnt.value, ctypes.byref(cnt), None, 0, ctypes.byref(nt)))
    bits = max([o.bits for o in ops[:cnt.value] if o.kind == 1], default=0)
    tab = np.zeros(max(1, nt.value) * 2 << bits, dtype=np.float64)
    _chk(lib().qs_plan_pass_ops(*args, ops, cnt.value, ctypes.byref(cnt), tab.ctypes.data, nt.value, ctypes.byref(nt)))
    out = []
    for o in ops[:cnt.value]:
        if o.kind == 1:
            out.append({"kind": 1, "table": o.table, "bits": o.bits,
                        "signs": [(o.sign_q[i], o.sign_t[i]) for i in range(o.nsigns)]})
        else:
            m = np.array(o.m[:]).view(np.complex128).reshape(2, 2)
            out.append({"kind": 0, "target": o.target, "ctrl_mask": o.ctrl_mask, "m": m})
    tables = tab.view(np.complex128).reshape(-1, 1 << bits)[:nt.value].copy()
    return out, tables


def qs_plan_passes(p: int) -> list:
    return [qs_plan_pass_info(p, i) for i in range(qs_plan_get_stats(p)["n_passes"])]


def qs_probs(h: int, qubits=None, out=None):
    """Marginal probabilities over `qubits` (default: all, in order).  `out` may be
    a device tensor (filled asynchronously) or omitted (returns numpy)."""
    n = qs_num_qubits(h)
    q = np.arange(n, dtype=np.int32) if qubits is None else np.ascontiguousarray(qubits, dtype=np.int32)
    if out is None:
        out = np.empty(1 << len(q), dtype=np.float64)
    ptr, dev = _host_or_dev(out)
    _chk(lib().qs_probs(h, q.ctypes.data if len(q) else None, len(q), ptr, dev))
    return out


def qs_probs_dict(h: int, qubits=None, threshold: float = 0.0) -> dict:
    n = qs_num_qubits(h)
    q = np.arange(n, dtype=np.int32) if qubits is None else np.ascontiguousarray(qubits, dtype=np.int32)
    cnt = ctypes.c_size_t()
    _chk(lib().qs_probs_dict(h, q.ctypes.data if len(q) else None, len(q), threshold, None, None, 0, ctypes.byref(cnt)))
    idx = np.empty(max(1, cnt.value), dtype=np.uint64)
    p = np.empty(max(1, cnt.value), dtype=np.float64)
    _chk(lib().qs_probs_dict(h, q.ctypes.data if len(q) else None, len(q), threshold, idx.ctypes.data,
                             p.ctypes.data, cnt.value, ctypes.byref(cnt)))
    width = len(q)
    return {format(int(i), f"0{width}b") if width else "": float(v) for i, v in zip(idx[:cnt.value], p[:cnt.value])}


def qs_expect_z_all(h: int) -> np.ndarray:
    out = np.empty(qs_num_qubits(h), dtype=np.float64)
    _chk(lib().qs_expect_z_all(h, out.ctypes.data))
    return out


def qs_expect_pauli(h: int, terms) -> float:
    t = as_paulis(terms)
    out = ctypes.c_double()
    _chk(lib().qs_expect_pauli(h, t.ctypes.data if len(t) else None, len(t), ctypes.byref(out)))
    return out.value


def qs_sample(h: int, seed: int, shots: int, out=None):
    if out is None:
        out = np.empty(shots, dtype=np.uint64)
    ptr, dev = _host_or_dev(out)
    _chk(lib().qs_sample(h, seed, shots, ptr, dev))
    return out


def qs_timing_enable(h: int, on: bool = True):
    _chk(lib().qs_timing_enable(h, 1 if on else 0))


def qs_timing_fetch(h: int) -> list[dict]:
    """Pending per-kernel timing records of the state (synchronises its stream)."""
    cnt = ctypes.c_size_t()
    cap = 1 << 16
    recs = []
    while True:
        buf = (TimingRecord * cap)()
        _chk(lib().qs_timing_fetch(h, buf, cap, ctypes.byref(cnt)))
        recs += [{k: getattr(buf[i], k) for k, _ in TimingRecord._fields_} for i in range(min(cnt.value, cap))]
        if cnt.value <= cap:
            return recs
        # more records than the buffer held: they were dropped; report it
        raise QsimError(-1, f"timing log held {cnt.value} records, more than {cap}")


def qs_launch_count() -> int:
    return int(lib().qs_launch_count())


PASS_FEATURES = 25


def qs_mlp_create(n_in: int, n_hidden: int, weights=None, seed: int = 0) -> int:
    h = ctypes.c_void_p()
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    _chk(lib().qs_mlp_create(n_in, n_hidden, None if w is None else w.ctypes.data, seed, ctypes.byref(h)))
    return h.value


def qs_mlp_free(m: int):
    _chk(lib().qs_mlp_free(m))


def qs_mlp_num_weights(m: int) -> int:
    n = ctypes.c_size_t()
    _chk(lib().qs_mlp_num_weights(m, ctypes.byref(n)))
    return n.value


def qs_mlp_get_weights(m: int) -> np.ndarray:
    w = np.empty(qs_mlp_num_weights(m), dtype=np.float64)
    _chk(lib().qs_mlp_get_weights(m, w.ctypes.data))
    return w


def qs_mlp_set_weights(m: int, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    _chk(lib().qs_mlp_set_weights(m, w.ctypes.data))


def qs_mlp_forward(m: int, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    B = x.shape[0]
    y = np.empty(B, dtype=np.float64)
    _chk(lib().qs_mlp_forward(m, x.ctypes.data, B, y.ctypes.data))
    return y


def qs_mlp_loss_grad(m: int, x, t):
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    loss = ctypes.c_double()
    g = np.empty(qs_mlp_num_weights(m), dtype=np.float64)
    _chk(lib().qs_mlp_loss_grad(m, x.ctypes.data, t.ctypes.data, x.shape[0], ctypes.byref(loss), g.ctypes.data))
    return loss.value, g


def qs_mlp_train(m: int, x, t, epochs: int, lr: float) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    loss = ctypes.c_double()
    _chk(lib().qs_mlp_train(m, x.ctypes.data, t.ctypes.data, x.shape[0], epochs, lr, ctypes.byref(loss)))
    return loss.value


def qs_plan_features(p: int, gates) -> np.ndarray:
    g = as_gates(gates)
    n = qs_plan_get_stats(p)["n_passes"]
    out = np.empty((max(n, 1), PASS_FEATURES), dtype=np.float64)
    _chk(lib().qs_plan_features(p, g.ctypes.data if len(g) else None, len(g), out.ctypes.data))
    return out[:n]


def qs_plan_create_learned(n: int, gates, model: int) -> int:
    g = as_gates(gates)
    h = ctypes.c_void_p()
    _chk(lib().qs_plan_create_learned(n, g.ctypes.data if len(g) else None, len(g), model, ctypes.byref(h)))
    return h.value


KOP_KINDS = 15


def qs_plan_pass_kernel_ops(p: int, i: int, gates, params=None):
    """(counts by kernel op kind, limb products per amplitude) of pass i."""
    g = as_gates(gates)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    counts = np.zeros(KOP_KINDS, dtype=np.int64)
    ipa = ctypes.c_double()
    _chk(lib().qs_plan_pass_kernel_ops(p, i, g.ctypes.data if len(g) else None, len(g),
                                       None if pr is None else pr.ctypes.data, counts.ctypes.data, ctypes.byref(ipa)))
    return counts, ipa.value


PASS_SCORER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t,
                               ctypes.POINTER(ctypes.c_double))


def qs_plan_create_scored(n: int, gates, score) -> int:
    """Learned-planner groupings with a host cost model: score(x) maps a
    (B, PASS_FEATURES) array of pass features to B predicted log(ms)."""
    g = as_gates(gates)

    def cb(_ctx, x, B, y):
        try:
            xs = np.ctypeslib.as_array(x, shape=(B * PASS_FEATURES,)).reshape(B, PASS_FEATURES).copy()
            np.ctypeslib.as_array(y, shape=(B,))[:] = np.asarray(score(xs), dtype=np.float64).reshape(B)
            return 0
        except Exception:
            return 1

    fn = PASS_SCORER(cb)
    h = ctypes.c_void_p()
    _chk(lib().qs_plan_create_scored(n, g.ctypes.data if len(g) else None, len(g),
                                     ctypes.cast(fn, ctypes.c_void_p), None, ctypes.byref(h)))
    return h.value


def qs_batch_create(n_per_set, gate_lists, n_params, term_lists) -> int:
    """Batch of sets: gate_lists[s] (records, param_idx relative to the set),
    n_params[s] parameters, term_lists[s] Pauli terms."""
    ns = len(n_per_set)
    nq = np.ascontiguousarray(n_per_set, dtype=np.int32)
    gates = as_gates(np.concatenate([as_gates(g) for g in gate_lists]) if ns else np.empty(0, GATE_DTYPE))
    terms = as_paulis(np.concatenate([as_paulis(t) for t in term_lists]) if ns else np.empty(0, PAULI_DTYPE))
    go = np.zeros(ns + 1, dtype=np.uint64)
    go[1:] = np.cumsum([len(g) for g in gate_lists])
    po = np.zeros(ns + 1, dtype=np.uint64)
    po[1:] = np.cumsum(n_params)
    to = np.zeros(ns + 1, dtype=np.uint64)
    to[1:] = np.cumsum([len(t) for t in term_lists])
    h = ctypes.c_void_p()
    _chk(lib().qs_batch_create(ns, nq.ctypes.data, gates.ctypes.data if len(gates) else None, go.ctypes.data,
                               po.ctypes.data, terms.ctypes.data if len(terms) else None, to.ctypes.data,
                               ctypes.byref(h)))
    return h.value


def qs_batch_run(b: int, params, energies=None, grads=None):
    """params: numpy (host path, CUDA graph) or CUDA tensor (device path)."""
    if energies is None:
        raise ValueError("energies output is required")
    pp, dev = _host_or_dev(params)
    ep, _ = _host_or_dev(energies)
    gp, _ = _host_or_dev(grads)
    _chk(lib().qs_batch_run(b, pp, ep, gp, dev))
    return energies, grads


def qs_batch_last_ms(b: int) -> float:
    ms = ctypes.c_double()
    _chk(lib().qs_batch_last_ms(b, ctypes.byref(ms)))
    return ms.value


def qs_batch_info(b: int) -> dict:
    g, t, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _chk(lib().qs_batch_info(b, ctypes.byref(g), ctypes.byref(t), ctypes.byref(s)))
    c = ctypes.c_int()
    _chk(lib().qs_batch_cluster(b, ctypes.byref(c)))
    return {"grid": g.value, "threads": t.value, "smem_bytes": s.value, "cluster": c.value}


def qs_batch_cluster(b: int) -> int:
    c = ctypes.c_int()
    _chk(lib().qs_batch_cluster(b, ctypes.byref(c)))
    return c.value


def qs_set_batch_cluster(ctas: int):
    _chk(lib().qs_set_batch_cluster(int(ctas)))


def qs_batch_free(b: int):
    _chk(lib().qs_batch_free(b))


def qs_adjoint_grad(h: int, gates, params, terms):
    """(energy, gradient) of <psi(params)|H|psi(params)>; overwrites the state."""
    g = as_gates(gates)
    pr = np.ascontiguousarray(params, dtype=np.float64)
    t = as_paulis(terms)
    e = ctypes.c_double()
    grad = np.empty(len(pr), dtype=np.float64)
    _chk(lib().qs_adjoint_grad(h, g.ctypes.data if len(g) else None, len(g), pr.ctypes.data if len(pr) else None,
                               len(pr), t.ctypes.data if len(t) else None, len(t), ctypes.byref(e),
                               grad.ctypes.data if len(pr) else None))
    return e.value, grad
