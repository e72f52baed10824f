"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *draws* inputs: gate programs (as packed records), angle vectors,
Pauli-sum descriptors and qubit counts.  It contains no gate matrix, no amplitude
arithmetic and no reduction, so neither side of a parity test can borrow method
arithmetic from it.

Record layout (56 bytes, little-endian, 8-byte aligned), the wire format both the
oracle and the CUDA library read:

    int32  type       gate code (GATE_CODES below)
    int32  q0         target of a 1-qubit gate; control of CNOT / CZ / CR
    int32  q1         target of CNOT / CZ / CR; -1 otherwise
    int32  param_idx  >= 0: theta is params[param_idx]; -1: theta is p[0]
    uint64 ctrl_mask  extra control qubits (bit q set: qubit q must be |1>)
    f64    p[3]       theta, phi, lambda
    int32  dagger     1: apply the adjoint of the gate
    int32  reserved   0

Pauli term layout (24 bytes): f64 coef, uint64 xmask, uint64 zmask; a qubit with
both bits set carries a Y.

Random draws use SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) with the double
mapping u = (x >> 11) * 2^-53, so the same seed gives the same program everywhere.
"""
from __future__ import annotations

import numpy as np

# Gate codes of the record format (the paper's gate set, Section "Structure of
# QPanda" keyword list and the "Performance of basic gates" experiment, plus P,
# the one-qubit phase gate that CR controls).
GATE_CODES = {
    "I": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "S": 5, "T": 6,
    "RX": 7, "RY": 8, "RZ": 9, "U3": 10, "P": 11,
    "CNOT": 12, "CZ": 13, "CR": 14,
}
ONE_QUBIT = ("H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "U3")
TWO_QUBIT = ("CNOT", "CZ", "CR")
ANGLED = ("RX", "RY", "RZ", "U3", "P", "CR")

GATE_DTYPE = np.dtype([
    ("type", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("param_idx", "<i4"),
    ("ctrl_mask", "<u8"), ("p", "<f8", (3,)), ("dagger", "<i4"), ("reserved", "<i4"),
], align=True)
assert GATE_DTYPE.itemsize == 56

PAULI_DTYPE = np.dtype([("coef", "<f8"), ("xmask", "<u8"), ("zmask", "<u8")], align=True)
assert PAULI_DTYPE.itemsize == 24

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    """Sequential SplitMix64 stream (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, k: int) -> int:
        """Integer in [0, k) (floor of a uniform double; k is small)."""
        return min(int(self.uniform() * k), k - 1)

    def angle(self) -> float:
        return self.uniform() * (2.0 * np.pi)


def gate(name: str, q0: int, q1: int = -1, theta: float = 0.0, phi: float = 0.0,
         lam: float = 0.0, ctrl_mask: int = 0, param_idx: int = -1, dagger: int = 0):
    """One record as a tuple in GATE_DTYPE field order."""
    return (GATE_CODES[name], q0, q1, param_idx, ctrl_mask, (theta, phi, lam), dagger, 0)


def pack(records) -> np.ndarray:
    return np.array(list(records), dtype=GATE_DTYPE)


def _distinct(rng: SplitMix64, n: int, k: int):
    out = []
    while len(out) < k:
        q = rng.below(n)
        if q not in out:
            out.append(q)
    return out


def _draw_gate(rng: SplitMix64, n: int, name: str):
    if name in TWO_QUBIT:
        c, t = _distinct(rng, n, 2)
        theta = rng.angle() if name == "CR" else 0.0
        return gate(name, c, t, theta=theta)
    (t,) = _distinct(rng, n, 1)
    if name == "U3":
        return gate(name, t, theta=rng.angle(), phi=rng.angle(), lam=rng.angle())
    if name in ANGLED:
        return gate(name, t, theta=rng.angle())
    return gate(name, t)


def random_circuit(n: int, n_gates: int, seed: int, two_qubit_prob: float | None = None) -> np.ndarray:
    """Random program over {H,X,Y,Z,S,T,RX,RY,RZ,U3,CNOT,CZ,CR}.

    two_qubit_prob None: each gate uniform over the 13 types.  Otherwise a gate is
    two-qubit with that probability (uniform over CNOT, CZ, CR) and else uniform over
    the ten one-qubit types.  Qubits are distinct and uniform (control drawn first);
    angles are uniform in [0, 2*pi).
    """
    rng = SplitMix64(seed)
    recs = []
    names13 = ONE_QUBIT + TWO_QUBIT
    for _ in range(n_gates):
        if n < 2:
            name = ONE_QUBIT[rng.below(len(ONE_QUBIT))]
        elif two_qubit_prob is None:
            name = names13[rng.below(len(names13))]
        elif rng.uniform() < two_qubit_prob:
            name = TWO_QUBIT[rng.below(3)]
        else:
            name = ONE_QUBIT[rng.below(len(ONE_QUBIT))]
        recs.append(_draw_gate(rng, n, name))
    return pack(recs)


def layered_u3_cz(n: int, depth: int, seed: int) -> np.ndarray:
    """Depth-`depth` layered circuit: U3(theta,phi,lambda ~ U[0,2pi)) on every qubit,
    then CZ on brickwork neighbour pairs -- (2j, 2j+1) on even layers, (2j+1, 2j+2)
    on odd layers.  n=30, depth=20 gives 600 U3 + 290 CZ."""
    rng = SplitMix64(seed)
    recs = []
    for layer in range(depth):
        for q in range(n):
            recs.append(gate("U3", q, theta=rng.angle(), phi=rng.angle(), lam=rng.angle()))
        start = 0 if layer % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            recs.append(gate("CZ", a, a + 1))
    return pack(recs)


def hea_ansatz(n: int, layers: int) -> tuple[np.ndarray, int]:
    """Hardware-efficient ansatz: per layer RY(theta) on every qubit, RZ(theta) on
    every qubit, then the CNOT ring CNOT(control=(i+1) mod n, target=i), i = 0..n-1.
    Every rotation reads its own parameter; returns (records, n_params)."""
    recs = []
    k = 0
    for _ in range(layers):
        for name in ("RY", "RZ"):
            for q in range(n):
                recs.append(gate(name, q, param_idx=k))
                k += 1
        if n >= 2:
            for i in range(n):
                c = (i + 1) % n
                if c != i:
                    recs.append(gate("CNOT", c, i))
    return pack(recs), k


def mixed_layers_circuit(n: int, layers: int, seed: int) -> tuple[np.ndarray, int]:
    """Parametrised layers mixing gate kinds: an H layer; per layer RY on every
    qubit (every third daggered), then per qubit one of RZ (on a parameter shared
    within the layer), P (alternately daggered), an unparametrised S, T or Z, or
    RZ on its own parameter, with one controlled RZ in the middle of the run; a
    CNOT ring (control (i+1) mod n, target i); H on even qubits.
    Returns (records, parameter count)."""
    rng = SplitMix64(seed)
    recs = [gate("H", qq) for qq in range(n)]
    p = 0
    for layer in range(layers):
        for qq in range(n):
            recs.append(gate("RY", qq, param_idx=p, dagger=int((qq + layer) % 3 == 0)))
            p += 1
        shared = p
        p += 1
        for qq in range(n):
            k = rng.below(5)
            if k == 0:
                recs.append(gate("RZ", qq, param_idx=shared))
            elif k == 1:
                recs.append(gate("P", qq, param_idx=p, dagger=qq & 1))
                p += 1
            elif k == 2:
                recs.append(gate(("S", "T", "Z")[rng.below(3)], qq))
            else:
                recs.append(gate("RZ", qq, param_idx=p))
                p += 1
            if qq == n // 2 and n > 1:
                recs.append(gate("RZ", qq, param_idx=p, ctrl_mask=1 << ((qq + 1) % n)))
                p += 1
        if n > 1:
            recs += [gate("CNOT", (qq + 1) % n, qq) for qq in range(n)]
        recs += [gate("H", qq) for qq in range(0, n, 2)]
    return pack(recs), p


def uniform_angles(count: int, seed: int) -> np.ndarray:
    rng = SplitMix64(seed)
    return np.array([rng.angle() for _ in range(count)], dtype=np.float64)


def zz_chain(n: int, coef: float = 1.0) -> np.ndarray:
    """sum_{i=0}^{n-2} Z_i Z_{i+1} (open chain)."""
    return np.array([(coef, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)], dtype=PAULI_DTYPE)


def tfim(n: int, h: float = 0.7) -> np.ndarray:
    """Transverse-field Ising, open chain: sum_i Z_i Z_{i+1} + h sum_i X_i."""
    zz = [(1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    xx = [(h, 1 << i, 0) for i in range(n)]
    return np.array(zz + xx, dtype=PAULI_DTYPE)


def random_paulis(n: int, n_terms: int, seed: int) -> np.ndarray:
    """Random Pauli strings with uniform coefficients in [-1, 1)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_terms):
        xm = zm = 0
        for q in range(n):
            k = rng.below(4)  # 0 I, 1 X, 2 Y, 3 Z
            if k in (1, 2):
                xm |= 1 << q
            if k in (2, 3):
                zm |= 1 << q
        out.append((2.0 * rng.uniform() - 1.0, xm, zm))
    return np.array(out, dtype=PAULI_DTYPE)


def batch_qubit_counts(n_sets: int, seed: int, lo: int = 10, hi: int = 20) -> np.ndarray:
    """Qubit count per parameter set, uniform over lo..hi inclusive."""
    rng = SplitMix64(seed)
    return np.array([lo + rng.below(hi - lo + 1) for _ in range(n_sets)], dtype=np.int32)


def random_state(n: int, seed: int) -> np.ndarray:
    """Unnormalised complex128 vector with entries uniform in [-1,1) x [-1,1)i,
    scaled by 2^{-n/2}; returned as interleaved float64 (re, im)."""
    rng = SplitMix64(seed)
    N = 1 << n
    v = np.empty(2 * N, dtype=np.float64)
    scale = 2.0 ** (-n / 2.0)
    for i in range(2 * N):
        v[i] = (2.0 * rng.uniform() - 1.0) * scale
    return v


def random_state_fast(n: int, seed: int) -> np.ndarray:
    """Same distribution as random_state but drawn with numpy's PCG64 (for large n)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return (g.random(2 << n) * 2.0 - 1.0) * 2.0 ** (-n / 2.0)


def random_matrix(k: int, seed: int) -> np.ndarray:
    """Dense 2^k x 2^k complex matrix (row-major, interleaved re/im), entries uniform
    in [-1,1) + [-1,1)i scaled by 2^{-k/2}; not unitary."""
    rng = SplitMix64(seed)
    d = 1 << k
    m = np.empty(2 * d * d, dtype=np.float64)
    for i in range(2 * d * d):
        m[i] = (2.0 * rng.uniform() - 1.0) * 2.0 ** (-k / 2.0)
    return m


# ---- programs with measurement and classical control ---------------------------------
# Instruction layout (56 bytes), read by the oracle and the CUDA library alike:
#   int32 op       PROGRAM_OPS
#   int32 qubit    MEASURE: measured qubit
#   int32 dst      MEASURE / ASSIGN: classical bit (int64 register) written
#   int32 alu      ASSIGN: CLASSICAL_OPS
#   int32 lhs, rhs operands: register index, or -1 for the immediate
#   int64 imm      the immediate
#   uint32 n_then  IF: length of the then-block that follows; WHILE: body length
#   uint32 n_else  IF: length of the else-block after the then-block; WHILE: 0
#   uint64 gate_begin, gate_end   GATES: range of the program's gate array
# IF and WHILE test their lhs operand for != 0; a WHILE re-tests before every pass.
PROGRAM_OPS = {"GATES": 0, "MEASURE": 1, "ASSIGN": 2, "IF": 3, "WHILE": 4}
CLASSICAL_OPS = {"MOV": 0, "ADD": 1, "SUB": 2, "MUL": 3, "DIV": 4, "AND": 5, "OR": 6, "XOR": 7,
                 "LT": 8, "LE": 9, "GT": 10, "GE": 11, "EQ": 12, "NE": 13, "NOT": 14}

PINSTR_DTYPE = np.dtype([
    ("op", "<i4"), ("qubit", "<i4"), ("dst", "<i4"), ("alu", "<i4"), ("lhs", "<i4"), ("rhs", "<i4"),
    ("imm", "<i8"), ("n_then", "<u4"), ("n_else", "<u4"), ("gate_begin", "<u8"), ("gate_end", "<u8"),
], align=True)
assert PINSTR_DTYPE.itemsize == 56


class Program:
    """Builder of a structured program: gate runs, measurements into classical
    registers, register assignments, if/else and while blocks (nested by length)."""

    def __init__(self):
        self.instrs = []
        self.gates = []

    def _emit(self, **kw):
        rec = dict(op=0, qubit=-1, dst=-1, alu=0, lhs=-1, rhs=-1, imm=0, n_then=0, n_else=0,
                   gate_begin=0, gate_end=0)
        rec.update(kw)
        self.instrs.append(rec)
        return len(self.instrs) - 1

    def apply(self, records):
        b = len(self.gates)
        self.gates.extend(list(np.asarray(records, dtype=GATE_DTYPE)))
        return self._emit(op=0, gate_begin=b, gate_end=len(self.gates))

    def measure(self, qubit: int, dst: int):
        return self._emit(op=1, qubit=qubit, dst=dst)

    def assign(self, dst: int, alu: str, lhs: int = -1, rhs: int = -1, imm: int = 0):
        return self._emit(op=2, dst=dst, alu=CLASSICAL_OPS[alu], lhs=lhs, rhs=rhs, imm=imm)

    def if_(self, cond: int, then_fn, else_fn=None):
        i = self._emit(op=3, lhs=cond)
        t0 = len(self.instrs)
        then_fn(self)
        t1 = len(self.instrs)
        if else_fn is not None:
            else_fn(self)
        self.instrs[i]["n_then"] = t1 - t0
        self.instrs[i]["n_else"] = len(self.instrs) - t1

    def while_(self, cond: int, body_fn):
        i = self._emit(op=4, lhs=cond)
        b0 = len(self.instrs)
        body_fn(self)
        self.instrs[i]["n_then"] = len(self.instrs) - b0

    def pack(self):
        prog = np.zeros(len(self.instrs), dtype=PINSTR_DTYPE)
        for k, rec in enumerate(self.instrs):
            for f, v in rec.items():
                prog[k][f] = v
        gates = np.array(self.gates, dtype=GATE_DTYPE) if self.gates else np.zeros(0, dtype=GATE_DTYPE)
        return prog, gates


def random_program(n: int, seed: int, segments: int = 6, gates_per_segment: int = 40, ncbits: int = 8):
    """Random structured program: gate runs drawn as random_circuit, measurements
    of random qubits, classical arithmetic on the registers, if/else on
    registers, and bounded while loops (a counter register caps each loop at 4
    passes).  Registers 0..ncbits-1; the last two are loop scratch."""
    rng = SplitMix64(seed)
    p = Program()
    cnt, flag = ncbits - 1, ncbits - 2
    data = ncbits - 2
    alus = ["MOV", "ADD", "SUB", "MUL", "DIV", "AND", "OR", "XOR", "LT", "LE", "GT", "GE", "EQ", "NE", "NOT"]

    def gates(pp):
        pp.apply(random_circuit(n, 1 + rng.below(gates_per_segment), rng.next_u64() & 0xFFFFFFFF))

    def measure(pp):
        pp.measure(rng.below(n), rng.below(data))

    def arith(pp):
        alu = alus[rng.below(len(alus))]
        if alu == "DIV":
            pp.assign(rng.below(data), alu, rng.below(data), -1, 1 + rng.below(3))
        elif rng.below(2):
            pp.assign(rng.below(data), alu, rng.below(data), rng.below(data))
        else:
            pp.assign(rng.below(data), alu, rng.below(data), -1, rng.below(5) - 2)

    def block(pp, depth):
        for _ in range(1 + rng.below(3)):
            k = rng.below(6 if depth < 2 else 3)
            if k == 0:
                gates(pp)
            elif k == 1:
                measure(pp)
            elif k == 2:
                arith(pp)
            elif k == 3:
                c = rng.below(data)
                if rng.below(2):
                    pp.if_(c, lambda q: block(q, depth + 1), lambda q: block(q, depth + 1))
                else:
                    pp.if_(c, lambda q: block(q, depth + 1))
            else:
                q = rng.below(n)

                def body(bb):
                    block(bb, depth + 1)
                    bb.assign(cnt, "ADD", cnt, -1, 1)
                    bb.measure(q, flag)
                    bb.assign(data - 1, "LT", cnt, -1, 4 * (depth + 1))
                    bb.assign(flag, "AND", flag, data - 1)
                pp.assign(flag, "MOV", -1, -1, 1)
                pp.while_(flag, body)

    for _ in range(segments):
        block(p, 0)
        gates(p)
    return p.pack()



# ---- noise rules -----------------------------------------------------------------------
# Rule layout (48 bytes): int32 model, int32 gate_type (-1: every gate), int32 q0,
# int32 q1 (the gate's first / second qubit, -1: any), f64 p, f64 t1, f64 t2, f64 tgate.
NOISE_MODELS = {"DAMPING": 0, "DEPHASING": 1, "DECOHERENCE": 2, "DEPOLARIZING": 3, "BITFLIP": 4,
                "BITPHASEFLIP": 5, "PHASEFLIP": 6, "PHASE_DAMPING": 7}
NOISE_DTYPE = np.dtype([("model", "<i4"), ("gate_type", "<i4"), ("q0", "<i4"), ("q1", "<i4"),
                        ("p", "<f8"), ("t1", "<f8"), ("t2", "<f8"), ("tgate", "<f8")], align=True)
assert NOISE_DTYPE.itemsize == 48


def noise_rule(model: str, gate: str | None = None, p: float = 0.0, q0: int = -1, q1: int = -1,
               t1: float = 0.0, t2: float = 0.0, tgate: float = 0.0):
    return (NOISE_MODELS[model], -1 if gate is None else GATE_CODES[gate], q0, q1, p, t1, t2, tgate)


def noise_rules(rules) -> np.ndarray:
    return np.array(list(rules), dtype=NOISE_DTYPE)
