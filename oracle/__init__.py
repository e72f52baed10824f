"""CPU oracle for the full-amplitude state-vector method (QPanda, arXiv 2212.14201).

TEST INFRASTRUCTURE ONLY.  The product package never imports this module; the test
suite, the smoke check and the benchmark's CPU-baseline leg do.  The arithmetic
lives in ``qsim_oracle.c`` (plain C, IEEE double, no fusion or tiling); this file
compiles it with gcc and wraps it with ctypes.

Every function states the paper passage it follows in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ELIMIT, EUNSUPPORTED = 0, -1, -2, -4, -5


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, OpenMP for the gate loop)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
            sig = {
                "or_gate_matrix": (i32, [P, i32, P, P, P, P]),
                "or_apply_gate": (i32, [P, i32, P, P]),
                "or_apply_circuit": (i32, [P, i32, P, i64, P]),
                "or_apply_matrix": (i32, [P, i32, P, i32, u64, P]),
                "or_init_zero": (None, [P, i32]),
                "or_probs": (None, [P, i32, P]),
                "or_marginal": (i32, [P, i32, P, i32, P]),
                "or_expect_z": (None, [P, i32, P]),
                "or_expect_pauli": (i32, [P, i32, P, i64, P]),
                "or_apply_pauli_sum": (i32, [P, i32, P, i64, P]),
                "or_splitmix64": (u64, [u64, u64]),
                "or_block_prefix": (i32, [P, i32, P]),
                "or_sample": (i32, [P, i32, u64, i64, P]),
                "or_adjoint_grad": (i32, [i32, P, i64, P, i64, P, i64, P, P]),
                "or_energy": (i32, [i32, P, i64, P, P, i64, P]),
                "or_mlp_nweights": (i64, [i32, i32]),
                "or_mlp_forward": (i32, [i32, i32, P, P, i64, P]),
                "or_mlp_loss_grad": (i32, [i32, i32, P, P, P, i64, P, P]),
                "or_measure": (i32, [P, i32, i32, ctypes.c_double, P, P]),
                "or_kraus": (i32, [i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P]),
                "or_run_noisy": (i32, [P, i32, P, i64, P, P, i64, ctypes.c_double, u64, P]),
                "or_readout": (None, [P, i64, i32, ctypes.c_double, ctypes.c_double, u64]),
                "or_dm_run": (i32, [P, i32, P, i64, P, P, i64]),
                "or_partial_amplitudes": (i32, [i32, P, i64, P, i32, P, i64, P, P]),
                "or_run_program": (i32, [P, i32, P, i64, P, i64, P, u64, u64, P, i64, P, i64, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _chk(rc: int, what: str):
    if rc != OK:
        raise OracleError(f"{what} failed with status {rc}")


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _state(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype == np.complex128:
        a = a.view(np.float64)
    assert a.dtype == np.float64
    return a


def zero_state(n: int) -> np.ndarray:
    """|0...0> as interleaved float64."""
    s = np.empty(2 << n, dtype=np.float64)
    _load().or_init_zero(s.ctypes.data, n)
    return s


def gate_matrix(g: np.ndarray, n: int, params=None):
    """(target, control mask, 2x2 complex matrix) of one record."""
    lib = _load()
    t = ctypes.c_int()
    cm = ctypes.c_uint64()
    m = np.empty(8, dtype=np.float64)
    g = np.ascontiguousarray(np.atleast_1d(g))
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    _chk(lib.or_gate_matrix(_ptr(g), n, _ptr(pr), ctypes.byref(t), ctypes.byref(cm), m.ctypes.data), "gate_matrix")
    return t.value, cm.value, m.view(np.complex128).reshape(2, 2)


def apply_circuit(state: np.ndarray, n: int, gates: np.ndarray, params=None) -> np.ndarray:
    """Apply every record in order, in place; returns the state."""
    state = _state(state)
    gates = np.ascontiguousarray(gates)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    _chk(_load().or_apply_circuit(state.ctypes.data, n, _ptr(gates), len(gates), _ptr(pr)), "apply_circuit")
    return state


def run(n: int, gates: np.ndarray, params=None) -> np.ndarray:
    """Final state of `gates` from |0...0> (interleaved float64)."""
    return apply_circuit(zero_state(n), n, gates, params)


def apply_matrix(state: np.ndarray, n: int, targets, mat: np.ndarray, ctrl_mask: int = 0) -> np.ndarray:
    state = _state(state)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    m = np.ascontiguousarray(mat)
    if m.dtype == np.complex128:
        m = m.view(np.float64)
    m = np.ascontiguousarray(m.reshape(-1), dtype=np.float64)
    _chk(_load().or_apply_matrix(state.ctypes.data, n, t.ctypes.data, len(t), ctrl_mask, m.ctypes.data), "apply_matrix")
    return state


def probs(state: np.ndarray, n: int) -> np.ndarray:
    state = _state(state)
    p = np.empty(1 << n, dtype=np.float64)
    _load().or_probs(state.ctypes.data, n, p.ctypes.data)
    return p


def marginal(state: np.ndarray, n: int, qubits) -> np.ndarray:
    state = _state(state)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    out = np.empty(1 << len(q), dtype=np.float64)
    _chk(_load().or_marginal(state.ctypes.data, n, q.ctypes.data, len(q), out.ctypes.data), "marginal")
    return out


def expect_z(state: np.ndarray, n: int) -> np.ndarray:
    state = _state(state)
    out = np.empty(n, dtype=np.float64)
    _load().or_expect_z(state.ctypes.data, n, out.ctypes.data)
    return out


def expect_pauli(state: np.ndarray, n: int, terms: np.ndarray) -> float:
    state = _state(state)
    terms = np.ascontiguousarray(terms)
    out = ctypes.c_double()
    _chk(_load().or_expect_pauli(state.ctypes.data, n, _ptr(terms), len(terms), ctypes.byref(out)), "expect_pauli")
    return out.value


def apply_pauli_sum(state: np.ndarray, n: int, terms: np.ndarray) -> np.ndarray:
    state = _state(state)
    terms = np.ascontiguousarray(terms)
    out = np.empty_like(state)
    _chk(_load().or_apply_pauli_sum(state.ctypes.data, n, _ptr(terms), len(terms), out.ctypes.data), "apply_pauli_sum")
    return out


def splitmix64(seed: int, s: int) -> int:
    return int(_load().or_splitmix64(seed, s))


def block_prefix(state: np.ndarray, n: int) -> np.ndarray:
    state = _state(state)
    L = min(1024, 1 << n)
    E = np.empty((1 << n) // L + 1, dtype=np.float64)
    _load().or_block_prefix(state.ctypes.data, n, E.ctypes.data)
    return E


def sample(state: np.ndarray, n: int, seed: int, shots: int) -> np.ndarray:
    state = _state(state)
    out = np.empty(shots, dtype=np.uint64)
    _chk(_load().or_sample(state.ctypes.data, n, seed, shots, out.ctypes.data), "sample")
    return out


def adjoint_grad(n: int, gates: np.ndarray, params: np.ndarray, terms: np.ndarray):
    """(energy, gradient) by the adjoint recursion."""
    gates = np.ascontiguousarray(gates)
    params = np.ascontiguousarray(params, dtype=np.float64)
    terms = np.ascontiguousarray(terms)
    e = ctypes.c_double()
    g = np.empty(len(params), dtype=np.float64)
    _chk(_load().or_adjoint_grad(n, _ptr(gates), len(gates), params.ctypes.data, len(params),
                                 _ptr(terms), len(terms), ctypes.byref(e), g.ctypes.data), "adjoint_grad")
    return e.value, g


def energy(n: int, gates: np.ndarray, params: np.ndarray, terms: np.ndarray) -> float:
    gates = np.ascontiguousarray(gates)
    params = np.ascontiguousarray(params, dtype=np.float64)
    terms = np.ascontiguousarray(terms)
    e = ctypes.c_double()
    _chk(_load().or_energy(n, _ptr(gates), len(gates), params.ctypes.data, _ptr(terms), len(terms),
                           ctypes.byref(e)), "energy")
    return e.value


def mlp_nweights(F: int, H: int) -> int:
    return int(_load().or_mlp_nweights(F, H))


def mlp_forward(F: int, H: int, w: np.ndarray, x: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, F)
    y = np.empty(len(x), dtype=np.float64)
    _chk(_load().or_mlp_forward(F, H, w.ctypes.data, x.ctypes.data, len(x), y.ctypes.data), "mlp_forward")
    return y


def mlp_loss_grad(F: int, H: int, w: np.ndarray, x: np.ndarray, t: np.ndarray):
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, F)
    t = np.ascontiguousarray(t, dtype=np.float64)
    loss = ctypes.c_double()
    g = np.empty_like(w)
    _chk(_load().or_mlp_loss_grad(F, H, w.ctypes.data, x.ctypes.data, t.ctypes.data, len(x), ctypes.byref(loss),
                                  g.ctypes.data), "mlp_loss_grad")
    return loss.value, g


def as_complex(state: np.ndarray) -> np.ndarray:
    return _state(state).view(np.complex128)


def measure(state: np.ndarray, n: int, qubit: int, u: float):
    """Projective measurement of one qubit with the draw u in [0, 1): returns
    (outcome, p1 / (p0 + p1), collapsed state)."""
    st = _state(state).copy()
    o = ctypes.c_int()
    p1 = ctypes.c_double()
    _chk(_load().or_measure(st.ctypes.data, n, qubit, u, ctypes.byref(o), ctypes.byref(p1)), "or_measure")
    return o.value, p1.value, st


def run_program(n: int, prog: np.ndarray, gates: np.ndarray, params=None, seed: int = 0,
                max_iters: int = 1 << 20, cbits=None, ncbits: int = 8, state=None, record_cap: int = 4096):
    """Runs a structured program (measurements, classical registers, if/while)
    from |0...0> (or `state`).  Returns (state, cbits, record of p1 per measurement)."""
    st = zero_state(n) if state is None else _state(state).copy()
    cb = np.zeros(ncbits, dtype=np.int64) if cbits is None else np.array(cbits, dtype=np.int64)
    rec = np.zeros(record_cap, dtype=np.float64)
    nm = ctypes.c_uint64()
    prog = np.ascontiguousarray(prog)
    gates = np.ascontiguousarray(gates)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    rc = _load().or_run_program(st.ctypes.data, n, _ptr(prog), len(prog), _ptr(gates) if len(gates) else None,
                                len(gates), _ptr(pr), seed, max_iters, cb.ctypes.data, len(cb), rec.ctypes.data,
                                record_cap, ctypes.byref(nm))
    _chk(rc, "or_run_program")
    return st, cb, rec[:min(nm.value, record_cap)].copy()


def kraus(model: int, p: float = 0.0, t1: float = 0.0, t2: float = 0.0, tgate: float = 0.0):
    """(list of 2x2 complex Kraus matrices, unital flag) of a noise model."""
    K = np.zeros(32, dtype=np.float64)
    un = ctypes.c_int()
    m = _load().or_kraus(model, p, t1, t2, tgate, K.ctypes.data, ctypes.byref(un))
    if m == 0:
        raise OracleError("or_kraus: bad noise model or parameters")
    Kc = K.view(np.complex128).reshape(4, 2, 2)[:m].copy()
    return list(Kc), bool(un.value)


def run_noisy(n: int, gates: np.ndarray, rules: np.ndarray, params=None, rot_err: float = 0.0, seed: int = 0,
              state=None):
    """One Monte-Carlo trajectory from |0...0> (or `state`): (state, draws used)."""
    st = zero_state(n) if state is None else _state(state).copy()
    gates = np.ascontiguousarray(gates)
    rules = np.ascontiguousarray(rules)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    nd = ctypes.c_uint64()
    rc = _load().or_run_noisy(st.ctypes.data, n, _ptr(gates) if len(gates) else None, len(gates), _ptr(pr),
                              _ptr(rules) if len(rules) else None, len(rules), rot_err, seed, ctypes.byref(nd))
    _chk(rc, "or_run_noisy")
    return st, nd.value


def readout(samples: np.ndarray, n: int, f0: float, f1: float, seed: int) -> np.ndarray:
    out = np.ascontiguousarray(samples, dtype=np.uint64).copy()
    _load().or_readout(out.ctypes.data, len(out), n, f0, f1, seed)
    return out


def dm_run(n: int, gates: np.ndarray, rules: np.ndarray, params=None) -> np.ndarray:
    """Density matrix after the noisy circuit (exact channel average), 2^n x 2^n."""
    N = 1 << n
    rho = np.empty(2 * N * N, dtype=np.float64)
    gates = np.ascontiguousarray(gates)
    rules = np.ascontiguousarray(rules)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    _chk(_load().or_dm_run(rho.ctypes.data, n, _ptr(gates) if len(gates) else None, len(gates), _ptr(pr),
                           _ptr(rules) if len(rules) else None, len(rules)), "or_dm_run")
    return rho.view(np.complex128).reshape(N, N)


def partial_amplitudes(n: int, gates: np.ndarray, n_low: int, indices, params=None):
    """Amplitudes <x|U|0...0> for the listed x by cutting the gates that cross the
    split (qubits < n_low | the rest): (complex array, number of paths)."""
    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    out = np.empty(2 * len(idx), dtype=np.float64)
    gates = np.ascontiguousarray(gates)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    npaths = ctypes.c_uint64()
    _chk(_load().or_partial_amplitudes(n, _ptr(gates) if len(gates) else None, len(gates), _ptr(pr), n_low,
                                       idx.ctypes.data, len(idx), out.ctypes.data, ctypes.byref(npaths)),
         "or_partial_amplitudes")
    return out.view(np.complex128).copy(), npaths.value
