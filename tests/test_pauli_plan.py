"""The pass planner of the exact Pauli sums (csrc/pauli_plan.h), compiled for the
host: structural invariants of every plan, and the planned passes evaluated with
exact Python integers over the Q60-rounded amplitudes against the oracle's plain
sum over x (the paper's expectation tool, Section "Variational quantum circuit")."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TMAX = SMAX = 12


@pytest.fixture(scope="module")
def pp():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "pauli_plan_check.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_2212_14201_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "pauli_plan_check.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.pp_plan.restype = ctypes.c_int
    lib.pp_plan.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
    return lib


def plan(pp, n, terms):
    nt = len(terms)
    xm = np.ascontiguousarray(terms["xmask"], dtype=np.uint64)
    zm = np.ascontiguousarray(terms["zmask"], dtype=np.uint64)
    cap_s, cap_p = 2 * nt + 1, 2 * nt + 2
    slots = np.zeros((cap_s, 3), dtype=np.int64)
    passes = np.zeros((cap_p, 2 + 2 * TMAX), dtype=np.int64)
    tm = np.zeros((max(nt, 1), 3), dtype=np.int32)
    ns, npa = ctypes.c_size_t(), ctypes.c_size_t()
    rc = pp.pp_plan(n, xm.ctypes.data, zm.ctypes.data, nt, slots.ctypes.data, cap_s, passes.ctypes.data, cap_p,
                    tm.ctypes.data, ctypes.byref(ns), ctypes.byref(npa))
    assert rc == 0
    sl = [(int(a) & (2**64 - 1), int(b) & (2**64 - 1), int(c)) for a, b, c in slots[:ns.value]]
    ps = []
    for r in passes[:npa.value]:
        T, k = int(r[0]), int(r[1])
        ps.append(([int(v) & (2**64 - 1) for v in r[2:2 + T]], [int(v) for v in r[2 + TMAX:2 + TMAX + k]]))
    return sl, ps, [tuple(int(v) for v in t) for t in tm[:nt]]


def lead(v):
    return v.bit_length() - 1


def coords(B, v):
    """Coordinates of v in the echelon basis B (None if v is outside the span)."""
    xc = 0
    for q in sorted(range(len(B)), key=lambda q: -lead(B[q])):
        if (v >> lead(B[q])) & 1:
            v ^= B[q]
            xc |= 1 << q
    return xc if v == 0 else None


def check_structure(n, terms, sl, ps, tm):
    seen = []
    for B, slots in ps:
        T = min(TMAX, n)
        assert len(B) == T and 1 <= len(slots) <= SMAX
        leads = [lead(b) for b in B]
        assert leads == sorted(leads) and len(set(leads)) == T  # echelon, ascending
        assert all(b < (1 << n) for b in B)
        assert B[:min(4, n)] == [1 << i for i in range(min(4, n))]  # runs of 16 consecutive amplitudes
        kinds = [sl[k][0] == 0 for k in slots]
        assert kinds == sorted(kinds, reverse=True)  # |a|^2 slots first
        keys = [(coords(B, sl[k][0]) << 1) | sl[k][2] for k in slots if sl[k][0]]
        assert None not in keys and keys == sorted(keys)  # pair slots in the span, grouped
        seen += slots
    assert sorted(seen) == list(range(len(sl)))  # every slot in exactly one pass
    for (coef, xm, zm), (s, t, m) in zip(terms, tm):
        xm, zm = int(xm), int(zm)
        ny = bin(xm & zm).count("1") & 3
        assert sl[s] == (xm, zm, ny & 1 if xm else 0)
        assert sl[t] == (xm, 0, ny & 1 if xm else 0)
        assert m == (1 if xm == 0 else (2 if ny in (0, 3) else -2))


def q60(v):
    return int(round(v * 2.0 ** 60))


def evaluate(n, psi, terms, sl, ps, tm):
    """The tile passes with exact integers: for each tile base (leading bits clear)
    and each slot, the sum of its values over entries or pairs of sign +1."""
    R = [q60(v) for v in psi[0::2]]
    I = [q60(v) for v in psi[1::2]]
    pos = {}
    for B, slots in ps:
        T = len(B)
        span = [0] * (1 << T)
        for e in range(1 << T):
            for i in range(T):
                if (e >> i) & 1:
                    span[e] ^= B[i]
        free = [b for b in range(n) if b not in {lead(v) for v in B}]
        for c in range(1 << (n - T)):
            base = sum(((c >> j) & 1) << b for j, b in enumerate(free))
            xs = [base ^ s for s in span]
            for k in slots:
                xm, zm, im = sl[k]
                acc = 0
                if xm == 0:
                    for x in xs:
                        if bin(x & zm).count("1") % 2 == 0:
                            acc += R[x] ** 2 + I[x] ** 2
                else:
                    xc = coords(B, xm)
                    top = lead(xc)
                    for e in range(1 << T):
                        if (e >> top) & 1:
                            continue
                        x0, x1 = xs[e], xs[e ^ xc]
                        assert x1 == x0 ^ xm
                        v = (R[x1] * I[x0] - I[x1] * R[x0]) if im else (R[x1] * R[x0] + I[x1] * I[x0])
                        if bin(x0 & zm).count("1") % 2 == 0:
                            acc += v
                pos[k] = pos.get(k, 0) + acc
    e = 0.0
    for (coef, _, _), (s, t, m) in zip(terms, tm):
        e += float(coef) * m * ((2 * pos[s] - pos[t]) / 2.0 ** 120)
    return e


def structured_terms(n):
    full = (1 << n) - 1
    rows = [(0.3, 0, 0)] + [(0.01 * (k + 1), 0, (k * 37 + 5) & full) for k in range(15)]
    shared = 0b101001 & full
    rows += [(0.02 * (k - 9), shared, (k * 11) & full) for k in range(17)]
    a, b = ((1 << (n - 1)) | 0b110) & full, ((1 << (n - 1)) | 0b011) & full
    rows += [(0.4, a, 0), (-0.25, b, (1 << (n - 1)) & full), (0.15, a ^ b, 0b101 & full)]
    for ny in range(4):
        ys = ((1 << ny) - 1) & full
        rows.append((0.1 * (ny + 1), ys | ((0b11 << (n - 2)) & full), ys))
    rows += [(-0.2, full, full), (0.05, full, 0)]
    return np.array(rows, dtype=w.PAULI_DTYPE)


@pytest.mark.parametrize("n,kind", [(1, "random"), (2, "structured"), (5, "random"), (7, "tfim"),
                                    (9, "structured"), (13, "tfim"), (14, "random")])
def test_plans_evaluate_to_the_oracle(pp, orc, n, kind):
    psi = w.random_state_fast(n, 60 + n)
    psi /= np.linalg.norm(psi)
    terms = {"random": lambda: w.random_paulis(n, 30, n), "structured": lambda: structured_terms(n),
             "tfim": lambda: w.tfim(n, 0.7)}[kind]()
    sl, ps, tm = plan(pp, n, terms)
    check_structure(n, terms, sl, ps, tm)
    assert abs(evaluate(n, psi, terms, sl, ps, tm) - orc.expect_pauli(psi, n, terms)) < 1e-12


@pytest.mark.parametrize("n", [30, 40, 64])
def test_plan_structure_at_size(pp, n):
    """The TFIM plan at the benchmark size (5 passes at n=30: tiles spanning 12, 8,
    8 and 2 of the X masks), and large random Hamiltonians, structure only."""
    tf = w.tfim(n, 0.7)
    sl, ps, tm = plan(pp, n, tf)
    check_structure(n, tf, sl, ps, tm)
    if n == 30:
        assert len(ps) == 5
        assert [sum(1 for k in s if sl[k][0]) for _, s in ps] == [12, 8, 8, 2, 0]
    rnd = w.random_paulis(n, 400, n + 1)
    sl, ps, tm = plan(pp, n, rnd)
    check_structure(n, rnd, sl, ps, tm)
