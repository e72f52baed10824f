"""Pins of the oracle's measurement, collapse and classical-control interpreter
(QMeasure / QIf / QWhile / ClassicalProg of the paper's Section "Core", and the
classical operators of Section "Qif and QWhile") against closed forms: the Born
rule, projective collapse, the paper's own QIf and QWhile examples, and integer
arithmetic."""
import math

import numpy as np
import pytest

import workloads as w

G = w.gate


def u01(seed, k, orc):
    return (orc.splitmix64(seed, k) >> 11) * 2.0 ** -53


def basis(n, x, amp=1.0):
    s = np.zeros(1 << n, dtype=np.complex128)
    s[x] = amp
    return s


def test_born_rule_and_collapse_single_qubit(orc):
    for theta in (0.3, 1.0, 2.5, math.pi / 2):
        st = orc.run(1, w.pack([G("RY", 0, theta=theta)]))
        p0 = math.cos(theta / 2) ** 2
        for u, want in ((p0 * (1 - 1e-9), 0), (p0 * (1 + 1e-9), 1), (0.0, 0), (1 - 2 ** -53, 1)):
            o, p1, post = orc.measure(st, 1, 0, u)
            assert o == want
            assert abs(p1 - math.sin(theta / 2) ** 2) < 1e-15
            c = orc.as_complex(post)
            assert abs(c[o] - 1.0) < 1e-15 and c[1 - o] == 0


def test_ghz_collapse(orc):
    for n in (3, 6):
        recs = [G("H", 0)] + [G("CNOT", i, i + 1) for i in range(n - 1)]
        st = orc.run(n, w.pack(recs))
        for q in range(n):
            for u in (0.25, 0.75):
                o, p1, post = orc.measure(st, n, q, u)
                assert abs(p1 - 0.5) < 1e-15
                assert o == (0 if u < 0.5 else 1)
                want = basis(n, 0 if o == 0 else (1 << n) - 1)
                assert np.max(np.abs(orc.as_complex(post) - want)) < 1e-15


def test_collapse_leaves_unmeasured_factor(orc):
    """|+> (x) psi, measuring qubit 0, gives |o> (x) psi (kron order: qubit 0 is
    the least significant bit)."""
    n = 5
    rest = orc.as_complex(orc.run(n - 1, w.random_circuit(n - 1, 40, 3)))
    plus = np.array([1, 1], dtype=np.complex128) / math.sqrt(2)
    st = np.kron(rest, plus)
    for u in (0.1, 0.9):
        o, p1, post = orc.measure(st, n, 0, u)
        e = np.zeros(2, dtype=np.complex128)
        e[o] = 1
        assert np.max(np.abs(orc.as_complex(post) - np.kron(rest, e))) < 1e-14
        # a second measurement repeats the outcome with certainty and changes nothing
        o2, p1b, post2 = orc.measure(post, n, 0, 0.5)
        assert o2 == o and p1b == float(o) and np.array_equal(post2, post)


def test_measurement_draws_follow_the_splitmix_stream(orc):
    """A program of MEASUREs uses draw k for measurement k: u_k = u01(SplitMix64
    number k), decided against the marginal of the current state."""
    n, seed = 4, 77
    gates = w.random_circuit(n, 30, 9)
    p = w.Program()
    p.apply(gates)
    for k in range(6):
        p.measure(k % n, k)
    prog, g = p.pack()
    st, cb, rec = orc.run_program(n, prog, g, seed=seed)
    ref = orc.run(n, gates)
    for k in range(6):
        o, p1, ref = orc.measure(ref, n, k % n, u01(seed, k, orc))
        assert cb[k] == o and rec[k] == p1
    assert np.array_equal(st, ref)


def paper_qif(c0, c1):
    p = w.Program()
    p.assign(2, "GT", 0, 1)
    p.if_(2, lambda q: q.apply([G("H", 0), G("H", 1), G("H", 2)]),
          lambda q: q.apply([G("H", 0), G("CNOT", 0, 1), G("CNOT", 1, 2)]))
    return p.pack()


def test_paper_qif_example(orc):
    """The paper's QIf listing: cbits[0]=0, cbits[1]=3, branch on cbits[0] >
    cbits[1]; the false branch builds GHZ_3, the true branch H on all three."""
    prog, g = paper_qif(0, 3)
    st, cb, _ = orc.run_program(3, prog, g, cbits=[0, 3, 0], ncbits=3)
    want = np.zeros(8, dtype=np.complex128)
    want[0] = want[7] = 1 / math.sqrt(2)
    assert np.max(np.abs(orc.as_complex(st) - want)) < 1e-15 and cb[2] == 0
    st, cb, _ = orc.run_program(3, prog, g, cbits=[5, 3, 0], ncbits=3)
    assert np.max(np.abs(orc.as_complex(st) - np.full(8, 1 / math.sqrt(8)))) < 1e-15 and cb[2] == 1


def test_paper_qwhile_example(orc):
    """The paper's QWhile listing: while cbits[1]: H on q0..q2, cbits[0] += 1,
    measure q1 into cbits[1].  Every measurement of q1 right after H has p1 =
    1/2, so the loop runs 1 + (number of leading draws >= 1/2) times; q1 ends in
    |0>, q0 and q2 in H^k |0> (up to a global sign: a 1 measured after H on |1>
    keeps the -1/sqrt(2) branch)."""
    p = w.Program()

    def body(b):
        b.apply([G("H", 0), G("H", 1), G("H", 2)])
        b.assign(0, "ADD", 0, -1, 1)
        b.measure(1, 1)
    p.while_(1, body)
    prog, g = p.pack()
    checked = 0
    for seed in range(40):
        us = [u01(seed, k, orc) for k in range(64)]
        if any(abs(u - 0.5) < 1e-9 for u in us):
            continue
        k = 1
        while us[k - 1] >= 0.5:
            k += 1
        st, cb, rec = orc.run_program(3, prog, g, seed=seed, cbits=[0, 1, 0], ncbits=3)
        assert cb[0] == k and cb[1] == 0 and len(rec) == k
        assert np.all(np.abs(rec - 0.5) < 1e-15)
        h = np.array([1, 1]) / math.sqrt(2) if k % 2 else np.array([1, 0])
        want = np.kron(h, np.kron(np.array([1, 0]), h)).astype(np.complex128)
        got = orc.as_complex(st)
        sign = np.sign(np.vdot(want, got).real)
        assert abs(sign) == 1 and np.max(np.abs(got - sign * want)) < 1e-15
        checked += 1
    assert checked > 30


def test_classical_operators(orc):
    g = np.random.Generator(np.random.PCG64(1))
    vals = [0, 1, -1, 2, -7, 13, 2 ** 62, -2 ** 63, 2 ** 63 - 1] + [int(x) for x in g.integers(-1000, 1000, 12)]
    M = 1 << 64

    def wrap(x):
        x %= M
        return x - M if x >= 1 << 63 else x

    def trunc_div(a, b):
        q = abs(a) // abs(b)
        return q if (a >= 0) == (b > 0) else -q
    ops = {"MOV": lambda a, b: a, "ADD": lambda a, b: wrap(a + b), "SUB": lambda a, b: wrap(a - b),
           "MUL": lambda a, b: wrap(a * b), "AND": lambda a, b: int(a != 0 and b != 0),
           "OR": lambda a, b: int(a != 0 or b != 0), "XOR": lambda a, b: wrap(a ^ b),
           "LT": lambda a, b: int(a < b), "LE": lambda a, b: int(a <= b), "GT": lambda a, b: int(a > b),
           "GE": lambda a, b: int(a >= b), "EQ": lambda a, b: int(a == b), "NE": lambda a, b: int(a != b),
           "NOT": lambda a, b: int(a == 0), "DIV": trunc_div}
    for name, f in ops.items():
        for a in vals:
            for b in vals[:10]:
                if name == "DIV" and (b == 0 or (a == -2 ** 63 and b == -1)):
                    continue
                p = w.Program()
                p.assign(2, name, 0, 1)
                prog, gg = p.pack()
                _, cb, _ = orc.run_program(1, prog, gg, cbits=[a, b, 0], ncbits=3)
                assert cb[2] == f(a, b), (name, a, b)
                # the immediate operand
                p = w.Program()
                p.assign(2, name, 0, -1, b)
                prog, gg = p.pack()
                _, cb, _ = orc.run_program(1, prog, gg, cbits=[a, 0, 0], ncbits=3)
                assert cb[2] == f(a, b), (name, a, b)


def test_errors_and_loop_bound(orc):
    p = w.Program()
    p.assign(0, "DIV", 1, -1, 0)
    prog, g = p.pack()
    with pytest.raises(orc.OracleError):
        orc.run_program(1, prog, g)
    p = w.Program()
    p.while_(-1, lambda b: b.apply([G("X", 0)]))   # condition: the immediate (0 by default)
    prog, g = p.pack()
    prog[0]["imm"] = 1                             # never false
    with pytest.raises(orc.OracleError):
        orc.run_program(1, prog, g, max_iters=100)
    prog[0]["n_then"] = 5                          # body beyond the program
    with pytest.raises(orc.OracleError):
        orc.run_program(1, prog, g)


def test_random_programs_are_normalised_and_deterministic(orc):
    for seed in range(6):
        prog, g = w.random_program(6, seed)
        a = orc.run_program(6, prog, g, seed=seed)
        b = orc.run_program(6, prog, g, seed=seed)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert abs(np.sum(a[0] ** 2) - 1.0) < 1e-13
        assert np.all((a[2] >= 0) & (a[2] <= 1))
