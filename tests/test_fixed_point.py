"""The Q60 fixed-point helpers the gate kernels use (csrc/fixed.h), compiled
for the host and checked against exact integer / rational arithmetic."""
import ctypes
import math
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fc():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "fixed_check.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_2212_14201_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "fixed_check.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.fc_from_double.restype = ctypes.c_longlong
    lib.fc_from_double.argtypes = [ctypes.c_double]
    lib.fc_from_double_nb.restype = ctypes.c_longlong
    lib.fc_from_double_nb.argtypes = [ctypes.c_double]
    lib.fc_dot2_exact.restype = None
    lib.fc_dot2_exact.argtypes = [ctypes.c_longlong] * 4 + [ctypes.c_void_p]
    lib.fc_to_double.restype = ctypes.c_double
    lib.fc_to_double.argtypes = [ctypes.c_longlong]
    lib.fc_to_double_nb.restype = ctypes.c_double
    lib.fc_to_double_nb.argtypes = [ctypes.c_longlong]
    lib.fc_pair_coef.restype = ctypes.c_int
    lib.fc_pair_coef.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.fc_triple_comp.restype = ctypes.c_int
    lib.fc_triple_comp.argtypes = [ctypes.c_void_p] * 5
    lib.fc_quad4_comp.restype = ctypes.c_int
    lib.fc_quad4_comp.argtypes = [ctypes.c_void_p] * 6
    lib.fc_add_rn_pos.restype = ctypes.c_double
    lib.fc_add_rn_pos.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
    lib.fc_sq_rn.restype = ctypes.c_double
    lib.fc_sq_rn.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
    lib.fc_pair_comp.restype = None
    lib.fc_pair_comp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.fc_dot2.restype = ctypes.c_longlong
    lib.fc_dot2.argtypes = [ctypes.c_longlong] * 4
    lib.fc_dot4.restype = ctypes.c_longlong
    lib.fc_dot4.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.fc_dot4_kernel.restype = ctypes.c_longlong
    lib.fc_dot4_kernel.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.fc_gauss_row.restype = None
    lib.fc_gauss_row.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.fc_dot4_full.restype = ctypes.c_longlong
    lib.fc_dot4_full.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    return lib


def exact_q60(v: float) -> int:
    """round(v * 2^60), ties away from zero, from the exact rational value."""
    f = Fraction(v) * (1 << 60)
    mag = abs(f)
    r = math.floor(mag + Fraction(1, 2))
    return r if f >= 0 else -r


def values(seed, count):
    g = np.random.Generator(np.random.PCG64(seed))
    v = list(g.uniform(-1.5, 1.5, count)) + list(g.uniform(-1, 1, count) * 2.0 ** -g.integers(0, 70, count))
    v += [0.0, -0.0, 1.0, -1.0, 1.5, -1.5, 2.0 ** -60, -2.0 ** -61, 2.0 ** -62, 3 * 2.0 ** -62, 5e-324,
          1 / math.sqrt(2), math.cos(1.0), 2.0 ** -8, 2.0 ** -8 * (1 + 2 ** -52)]
    return v


def test_from_double_is_correctly_rounded(fc):
    for v in values(1, 3000):
        assert fc.fc_from_double(v) == exact_q60(v), v


def test_branch_free_decode_matches(fc):
    """q60_from_double_nb: the same rounding for every exponent |v| < 8 can have,
    the largest values, ties, zeros and subnormals."""
    vs = values(2, 3000)
    for e in range(-75, 3):
        for m in (1.0, 1.5, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52):
            vs += [m * 2.0 ** e, -m * 2.0 ** e]
    vs += [7.999999999999999, -7.999999999999999, 2.0 ** -61 * 3, 2.0 ** -63, 2.0 ** -62, -(2.0 ** -62),
           2.0 ** -62 * (1 + 2.0 ** -52), 5e-324, -5e-324, 2.2250738585072014e-308]
    for v in vs:
        assert fc.fc_from_double_nb(v) == exact_q60(v), v


def test_exact_pair_products(fc):
    """split31 / dot2_exact: x1 y1 + x2 y2 exactly (modulo 2^128) over the whole
    range |v| < 2^61, including the extremes of every column sum."""
    g = np.random.Generator(np.random.PCG64(5))
    lim = (1 << 61) - 1
    edge = [lim, -lim, (1 << 60) + (1 << 30), -(1 << 30), (1 << 30) - 1, 0, 1, -1, (1 << 31) + (1 << 30)]
    cases = [tuple(int(x) for x in g.integers(-lim, lim, 4, dtype=np.int64)) for _ in range(3000)]
    cases += [(a, b, c, d) for a in edge for b in edge for c in edge[:3] for d in edge[:3]]
    out = (ctypes.c_ulonglong * 2)()
    for x1, y1, x2, y2 in cases:
        fc.fc_dot2_exact(x1, y1, x2, y2, out)
        want = (x1 * y1 + x2 * y2) % (1 << 128)
        assert out[0] + (out[1] << 64) == want, (x1, y1, x2, y2)


def test_to_double_is_correctly_rounded(fc):
    g = np.random.Generator(np.random.PCG64(2))
    Vs = [int(x) for x in g.integers(-(1 << 61), 1 << 61, 3000, dtype=np.int64)]
    Vs += [int(x) >> int(s) for x, s in zip(g.integers(-(1 << 61), 1 << 61, 2000, dtype=np.int64),
                                            g.integers(0, 60, 2000))]
    Vs += [0, 1, -1, 2, (1 << 53) + 1, (1 << 54) + 2, (1 << 54) + 6, (1 << 60), -(1 << 60), (1 << 61) - 1]
    for V in Vs:
        got = fc.fc_to_double(V)
        want = float(Fraction(V, 1 << 60))   # Python's int/Fraction -> float is correctly rounded (half even)
        assert got == want, V


def test_roundtrip_exact_for_large_values(fc):
    for v in values(3, 2000):
        if abs(v) >= 2.0 ** -8:
            assert fc.fc_to_double(fc.fc_from_double(v)) == v


def unitary_row(g):
    """Real and imaginary parts of one row of a random 2x2 unitary, as Q60
    integers (their absolute values sum to at most 2)."""
    z = g.normal(size=2) + 1j * g.normal(size=2)
    z /= np.linalg.norm(z)
    return [int(round(v * (1 << 60))) for v in (z[0].real, -z[0].imag, z[1].real, -z[1].imag)]


def test_limb_products_error_bound(fc):
    g = np.random.Generator(np.random.PCG64(4))
    for _ in range(3000):
        u = unitary_row(g)
        a = [int(x) for x in g.integers(-int(1.25 * (1 << 60)), int(1.25 * (1 << 60)), 4, dtype=np.int64)]
        exact = Fraction(sum(x * y for x, y in zip(u, a)), 1 << 60)
        ua = (ctypes.c_longlong * 4)(*u)
        aa = (ctypes.c_longlong * 4)(*a)
        got = fc.fc_dot4(ua, aa)
        assert fc.fc_dot4_kernel(ua, aa) == got   # pre-biased accumulator: identical value
        # four dropped low-limb products (< 2^60 each in 2^-120 units -> < 1 in Q60 units) + rounding
        assert abs(got - exact) <= 4 + 1
        got2 = fc.fc_dot2(u[0], a[0], u[1], a[1])
        assert abs(got2 - Fraction(u[0] * a[0] + u[1] * a[1], 1 << 60)) <= 2 + 1


def test_full_limb_products_are_correctly_rounded(fc):
    """The inner-product accumulator keeps all four limb products: its result is
    the exact sum rounded to the nearest multiple of 2^-60 (ties upward), with no
    bias to accumulate over 2^n terms."""
    g = np.random.Generator(np.random.PCG64(5))
    errs = []
    for _ in range(3000):
        u = [int(x) for x in g.integers(-(1 << 59), 1 << 59, 4, dtype=np.int64)]
        a = [int(x) for x in g.integers(-int(1.25 * (1 << 60)), int(1.25 * (1 << 60)), 4, dtype=np.int64)]
        exact = Fraction(sum(x * y for x, y in zip(u, a)), 1 << 60)
        got = fc.fc_dot4_full((ctypes.c_longlong * 4)(*u), (ctypes.c_longlong * 4)(*a))
        assert abs(got - exact) <= Fraction(1, 2)
        errs.append(float(got - exact))
    assert abs(np.mean(errs)) < 0.05


def test_extreme_limbs_do_not_overflow(fc):
    M = int(1.25 * (1 << 60))
    h = 1 << 59   # four entries of 1/2: the largest sum of absolute values a unitary row allows
    for u in ([h] * 4, [-h] * 4, [h, -h, h, -h]):
        for a in ([M] * 4, [-M] * 4, [M, -M, M, -M], [M - 1] * 4):
            ua = (ctypes.c_longlong * 4)(*u)
            aa = (ctypes.c_longlong * 4)(*a)
            exact = Fraction(sum(x * y for x, y in zip(u, a)), 1 << 60)
            assert abs(fc.fc_dot4(ua, aa) - exact) <= 5


def test_gauss_row_error_bound(fc):
    """A general 2x2 row in the three-product (Gauss) form: u0 a0 + u1 a1 for a
    row of a random unitary and amplitudes of modulus up to 1.25 (the Q60 state
    bound), against exact rational arithmetic on the same Q60-rounded inputs:
    six dropped low-limb products plus the final rounding."""
    g = np.random.Generator(np.random.PCG64(6))
    for trial in range(3000):
        z = g.normal(size=2) + 1j * g.normal(size=2)
        z /= np.linalg.norm(z)
        u = [z[0].real, z[0].imag, z[1].real, z[1].imag]
        amp = g.normal(size=2) + 1j * g.normal(size=2)
        amp *= 1.25 / np.abs(amp) if trial % 3 == 0 else 1.0 / max(1.0, np.max(np.abs(amp)))
        a = [int(round(v * (1 << 60))) for v in (amp[0].real, amp[0].imag, amp[1].real, amp[1].imag)]
        a = [max(min(v, int(1.25 * (1 << 60))), -int(1.25 * (1 << 60))) for v in a]
        out = (ctypes.c_longlong * 2)()
        fc.fc_gauss_row((ctypes.c_double * 4)(*u), (ctypes.c_longlong * 4)(*a), out)
        uq = [fc.fc_from_double(v) for v in u]
        ex_re = Fraction(uq[0] * a[0] - uq[1] * a[1] + uq[2] * a[2] - uq[3] * a[3], 1 << 60)
        ex_im = Fraction(uq[0] * a[1] + uq[1] * a[0] + uq[2] * a[3] + uq[3] * a[2], 1 << 60)
        assert abs(out[0] - ex_re) <= 7, trial
        assert abs(out[1] - ex_im) <= 7, trial


def test_branch_free_to_double_matches(fc):
    """The branch-free conversion the register engine uses gives the same double
    as the reference conversion (itself checked against exact rounding above)."""
    g = np.random.Generator(np.random.PCG64(11))
    Vs = [0, 1, -1, 2 ** 53 - 1, 2 ** 53, 2 ** 53 + 1, -(2 ** 53 + 3), 2 ** 60, -(2 ** 60), 2 ** 61 + 5, -(2 ** 61) - 7]
    Vs += [int(x) for x in g.integers(-2 ** 61, 2 ** 61, 4000)]
    Vs += [int(x) >> int(k) for x, k in zip(g.integers(-2 ** 61, 2 ** 61, 2000), g.integers(0, 61, 2000))]
    # ties at the 53-bit boundary: both parities of the kept bit
    Vs += [(m << 11) | 0x400 for m in range(2 ** 52, 2 ** 52 + 8)] + [-((m << 10) | 0x200) for m in range(2 ** 52, 2 ** 52 + 8)]
    for V in Vs:
        assert fc.fc_to_double_nb(V) == fc.fc_to_double(V), V


def _orth(g, reflect):
    t = g.uniform(0, 2 * np.pi)
    c, s = math.cos(t), math.sin(t)
    return np.array([c, s, s, -c] if reflect else [c, -s, s, c], dtype=np.float64)


@pytest.mark.parametrize("fa,fb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_pair_as_two_complex_products(fc, fa, fb):
    """R_b (x) R_a on a quad component through the two-complex-product form.
    (1) The coefficients: u = z0 + i z1 and v = z0 - i z1 (z_b = x_b0 + i x_b1,
    after the reflections' sign flips) scaled by P and Q, then z0 = u' + v',
    z1 = -i (u' - v'), reproduce the 4x4 Kronecker product of the two double
    matrices within double rounding.  (2) The limb arithmetic: the kernel's
    outputs equal that formula evaluated exactly on the same Q60 integers (inputs
    and the kernel's rounded P, Q) within 12 units of 2^-60."""
    g = np.random.Generator(np.random.PCG64(20 + 2 * fa + fb))
    sa, sb = (-1 if fa else 1), (-1 if fb else 1)
    for _ in range(300):
        ra, rb = _orth(g, fa), _orth(g, fb)
        c = np.zeros(6, dtype=np.int64)
        flags = fc.fc_pair_coef(ra.ctypes.data, rb.ctypes.data, c.ctypes.data)
        assert flags == fa | (fb << 1)
        P = complex(c[0], c[1]) / 2.0 ** 60
        Q = complex(c[3], c[4]) / 2.0 ** 60
        assert c[2] == -c[1] and c[5] == -c[4]

        # (1) the matrix of the form, column by column, against kron(rb, ra)
        K = np.kron(rb.reshape(2, 2), ra.reshape(2, 2))
        for qi in range(4):
            e = np.zeros(4)
            e[qi] = 1.0
            y = [e[0], sa * e[1], sb * e[2], sa * sb * e[3]]
            u = complex(y[0] - y[3], y[1] + y[2])
            v = complex(y[0] + y[3], y[1] - y[2])
            U, V = P * u, Q * v
            col = [U.real + V.real, U.imag + V.imag, U.imag - V.imag, V.real - U.real]
            assert np.max(np.abs(np.array(col) - K[:, qi])) < 4e-16
        # (2) the limb arithmetic against the exact evaluation on the same integers
        v = g.normal(size=4)
        v *= g.uniform(0, 1.25) / np.linalg.norm(v)
        x = np.array([exact_q60(float(t)) for t in v], dtype=np.int64)
        out = x.copy()
        fc.fc_pair_comp(ra.ctypes.data, rb.ctypes.data, out.ctypes.data)
        y = [Fraction(int(x[0])), sa * Fraction(int(x[1])), sb * Fraction(int(x[2])), sa * sb * Fraction(int(x[3]))]
        ur, ui = y[0] - y[3], y[1] + y[2]
        vr, vi = y[0] + y[3], y[1] - y[2]
        pr, pi, qr, qi_ = (Fraction(int(t), 1 << 60) for t in (c[0], c[1], c[3], c[4]))
        Ur, Ui = pr * ur - pi * ui, pi * ur + pr * ui
        Vr, Vi = qr * vr - qi_ * vi, qi_ * vr + qr * vi
        exact = [Ur + Vr, Ui + Vi, Ui - Vi, Vr - Ur]
        for qo in range(4):
            assert abs(Fraction(int(out[qo])) - exact[qo]) <= 12, (qo, float(Fraction(int(out[qo])) - exact[qo]))


@pytest.mark.parametrize("flags", range(8))
def test_triple_as_four_complex_products(fc, flags):
    """R_c (x) R_b (x) R_a on an octet component through the four-complex-product
    form (every combination of rotations and reflections): (1) the coefficients
    reproduce the 8x8 Kronecker product of the double matrices within double
    rounding; (2) the limb arithmetic equals the formula evaluated exactly on the
    same Q60 integers within 20 units of 2^-60."""
    g = np.random.Generator(np.random.PCG64(40 + flags))
    sg = [(-1 if (flags >> i) & 1 else 1) for i in range(3)]
    for _ in range(200):
        rs = [_orth(g, (flags >> i) & 1) for i in range(3)]
        v = g.normal(size=8)
        v *= g.uniform(0, 1.25) / np.linalg.norm(v)
        x = np.array([exact_q60(float(t)) for t in v], dtype=np.int64)
        out = x.copy()
        c = np.zeros(8, dtype=np.int64)
        got_flags = fc.fc_triple_comp(rs[0].ctypes.data, rs[1].ctypes.data, rs[2].ctypes.data, out.ctypes.data,
                                      c.ctypes.data)
        assert got_flags == flags

        def form(y, P, mul, add):
            ur = [y[4 * k] - y[4 * k + 3] for k in (0, 1)]
            ui = [y[4 * k + 1] + y[4 * k + 2] for k in (0, 1)]
            vr = [y[4 * k] + y[4 * k + 3] for k in (0, 1)]
            vi = [y[4 * k + 1] - y[4 * k + 2] for k in (0, 1)]
            Y = [(ur[0] - ui[1], ui[0] + ur[1]), (ur[0] + ui[1], ui[0] - ur[1]),
                 (vr[0] - vi[1], vi[0] + vr[1]), (vr[0] + vi[1], vi[0] - vr[1])]
            R = [(mul(P[k][0], Y[k][0]) - mul(P[k][1], Y[k][1]), mul(P[k][1], Y[k][0]) + mul(P[k][0], Y[k][1]))
                 for k in range(4)]
            u0 = (R[0][0] + R[1][0], R[0][1] + R[1][1]); u1 = (R[0][1] - R[1][1], R[1][0] - R[0][0])
            v0 = (R[2][0] + R[3][0], R[2][1] + R[3][1]); v1 = (R[2][1] - R[3][1], R[3][0] - R[2][0])
            res = []
            for u, w in ((u0, v0), (u1, v1)):
                res += [u[0] + w[0], u[1] + w[1], u[1] - w[1], w[0] - u[0]]
            return res

        # (1) columns of the form against kron(rc, kron(rb, ra))
        K = np.kron(rs[2].reshape(2, 2), np.kron(rs[1].reshape(2, 2), rs[0].reshape(2, 2)))
        P = [(c[2 * k] / 2.0 ** 60, c[2 * k + 1] / 2.0 ** 60) for k in range(4)]
        for qi in range(8):
            y = [0.0] * 8
            y[qi] = float(sg[0] ** (qi & 1) * sg[1] ** ((qi >> 1) & 1) * sg[2] ** ((qi >> 2) & 1))
            col = form(y, P, lambda a, b: a * b, None)
            assert np.max(np.abs(np.array(col) - K[:, qi])) < 6e-16, qi
        # (2) limb arithmetic against the exact evaluation on the same integers
        y = [Fraction(int(x[k])) * (sg[0] ** (k & 1) * sg[1] ** ((k >> 1) & 1) * sg[2] ** ((k >> 2) & 1)) for k in range(8)]
        Pq = [(Fraction(int(c[2 * k]), 1 << 60), Fraction(int(c[2 * k + 1]), 1 << 60)) for k in range(4)]
        exact = form(y, Pq, lambda a, b: a * b, None)
        for k in range(8):
            assert abs(Fraction(int(out[k])) - exact[k]) <= 20, (k, float(Fraction(int(out[k])) - exact[k]))


def _form4(y, P, mul):
    """R_d (x) R_c (x) R_b (x) R_a on one component of 16 values through eight
    complex products: pairs along a as complex numbers, the basis change
    (lo, hi) -> (lo + i hi, lo - i hi) along b, c, d, channel k times P[k], and
    the inverse (A, B) -> (A + B, -i (A - B)); values as (re, im) pairs."""
    z = [(y[2 * j], y[2 * j + 1]) for j in range(8)]
    for bit in (1, 2, 4):
        for j in range(8):
            if not j & bit:
                (lr, li), (hr, hi) = z[j], z[j | bit]
                z[j], z[j | bit] = (lr - hi, li + hr), (lr + hi, li - hr)
    z = [(mul(P[k][0], z[k][0]) - mul(P[k][1], z[k][1]), mul(P[k][1], z[k][0]) + mul(P[k][0], z[k][1]))
         for k in range(8)]
    for bit in (4, 2, 1):
        for j in range(8):
            if not j & bit:
                (ar, ai), (br, bi) = z[j], z[j | bit]
                z[j], z[j | bit] = (ar + br, ai + bi), (ai - bi, br - ar)
    out = []
    for re, im in z:
        out += [re, im]
    return out


@pytest.mark.parametrize("flags", [0, 1, 6, 9, 15])
def test_quad4_as_eight_complex_products(fc, flags):
    """Four rotations or reflections on one component of 16 amplitudes through the
    eight-complex-product form: (1) the coefficients reproduce the 16x16 Kronecker
    product of the double matrices within double rounding; (2) the limb arithmetic
    equals the form evaluated exactly on the same Q60 integers within 36 units of
    2^-60 (eight rounded products per output)."""
    g = np.random.Generator(np.random.PCG64(70 + flags))
    sg = [(-1 if (flags >> i) & 1 else 1) for i in range(4)]

    def sgn(k):
        return sg[0] ** (k & 1) * sg[1] ** ((k >> 1) & 1) * sg[2] ** ((k >> 2) & 1) * sg[3] ** ((k >> 3) & 1)
    for _ in range(100):
        rs = [_orth(g, (flags >> i) & 1) for i in range(4)]
        v = g.normal(size=16)
        v *= g.uniform(0, 1.25) / np.linalg.norm(v)
        x = np.array([exact_q60(float(t)) for t in v], dtype=np.int64)
        out = x.copy()
        c = np.zeros(16, dtype=np.int64)
        got_flags = fc.fc_quad4_comp(rs[0].ctypes.data, rs[1].ctypes.data, rs[2].ctypes.data, rs[3].ctypes.data,
                                     out.ctypes.data, c.ctypes.data)
        assert got_flags == flags
        # (1) columns of the form against kron(rd, kron(rc, kron(rb, ra)))
        K = np.kron(rs[3].reshape(2, 2), np.kron(rs[2].reshape(2, 2), np.kron(rs[1].reshape(2, 2),
                                                                               rs[0].reshape(2, 2))))
        P = [(c[2 * k] / 2.0 ** 60, c[2 * k + 1] / 2.0 ** 60) for k in range(8)]
        for qi in range(16):
            y = [0.0] * 16
            y[qi] = float(sgn(qi))
            col = _form4(y, P, lambda a, b: a * b)
            assert np.max(np.abs(np.array(col) - K[:, qi])) < 1e-15, qi
        # (2) limb arithmetic against the exact evaluation on the same integers
        y = [Fraction(int(x[k])) * sgn(k) for k in range(16)]
        Pq = [(Fraction(int(c[2 * k]), 1 << 60), Fraction(int(c[2 * k + 1]), 1 << 60)) for k in range(8)]
        exact = _form4(y, Pq, lambda a, b: a * b)
        for k in range(16):
            assert abs(Fraction(int(out[k])) - exact[k]) <= 36, (k, float(Fraction(int(out[k])) - exact[k]))


def test_integer_square_is_ieee_multiplication(fc):
    """The sampler's squares from integer operations equal IEEE 754 binary64
    multiplication x * x (round to nearest, ties to even) bit for bit: random
    significands over the whole valid exponent range, both signs, zero, the range
    ends, products just below and at a power of two, and exact ties (a significand
    of 27 significant bits whose square has a set round bit and no sticky bits)."""
    g = np.random.Generator(np.random.PCG64(91))
    xs = [0.0, -0.0, 1.0, -1.0, 2.0 ** -511, 2.0 ** 511 * (1 - 2.0 ** -53), 1.25, 0.7071067811865476,
          np.nextafter(np.sqrt(2.0), 0.0), np.sqrt(2.0), np.nextafter(1.0, 2.0), np.nextafter(2.0, 0.0)]
    xs += list(g.uniform(-1.5, 1.5, size=20000))
    xs += list(g.uniform(1.0, 2.0, size=20000) * 2.0 ** g.integers(-511, 511, size=20000).astype(np.float64))
    xs += list(2.0 ** -15 * g.normal(size=20000))
    ties = 0
    for k in range(1, 4000, 2):                       # odd 27-bit significands above 2^26.5
        m = (1 << 27) - k
        x = float(m) * 2.0 ** -26 * (1.0 if k % 3 else 2.0 ** -200)
        xs.append(x)
        p = m * m                                     # exact square
        top = p.bit_length() - 1
        sh = top - 52
        if sh > 0 and (p >> (sh - 1)) & 1 and p & ((1 << (sh - 1)) - 1) == 0:
            ties += 1
    assert ties > 100
    ok = ctypes.c_int()
    for x in xs:
        x = float(x)
        got = fc.fc_sq_rn(x, ctypes.byref(ok))
        assert ok.value == 1, x
        want = np.float64(x) * np.float64(x)
        assert np.float64(got).view(np.uint64) == want.view(np.uint64), (x, got, want)
    for x in (2.0 ** -512, 2.0 ** -600, 5e-324, 2.0 ** 512, float("inf")):
        fc.fc_sq_rn(x, ctypes.byref(ok))
        assert ok.value == 0, x


def test_integer_sum_is_ieee_addition(fc):
    """fl(a + b) of non-negative doubles from integer operations equals IEEE 754
    binary64 addition bit for bit: exponent differences 0..70 in both orders,
    zeros, exact ties below an even and an odd significand, carries into the next
    binade, and squares of amplitudes as the sampler forms them."""
    g = np.random.Generator(np.random.PCG64(92))
    pairs = [(0.0, 0.0), (0.0, 1.5), (2.0 ** -52, 0.0), (1.0, 2.0 ** -53), (1.0 + 2.0 ** -52, 2.0 ** -53),
             (1.0, 3 * 2.0 ** -53), (np.nextafter(2.0, 0.0), 2.0 ** -53), (np.nextafter(2.0, 0.0), 2.0 ** -52),
             (1.0, 1.0), (1.5, 1.5), (2.0 ** 1000, 2.0 ** 1000), (1.0, 2.0 ** -1000),
             (1.0, 2.0 ** -53 * (1 + 2.0 ** -52)), (1.0 + 2.0 ** -52, 2.0 ** -53 * (1 + 2.0 ** -52)),
             (1.0, 2.0 ** -53 * (1 - 2.0 ** -53))]  # half an ulp plus / minus a sticky bit
    for d in range(0, 71):
        a = g.uniform(1.0, 2.0, size=300) * 2.0 ** g.integers(-300, 300, size=300)
        b = g.uniform(1.0, 2.0, size=300) * a * 2.0 ** -d
        pairs += list(zip(a, b)) + list(zip(b, a))
        # ties: b exactly half an ulp of a (times an odd integer below 2^10)
        for k in (1, 3, 5, 1023):
            pairs.append((a[0], k * np.spacing(a[0]) / 2.0 ** min(d, 10)))
    v = 2.0 ** -15 * g.normal(size=(20000, 2))
    pairs += [(x * x, y * y) for x, y in v]
    ok = ctypes.c_int()
    for a, b in pairs:
        a, b = float(a), float(b)
        got = fc.fc_add_rn_pos(a, b, ctypes.byref(ok))
        assert ok.value == 1, (a, b)
        want = np.float64(a) + np.float64(b)
        assert np.float64(got).view(np.uint64) == want.view(np.uint64), (a, b, got, want)
    for a, b in ((-1.0, 1.0), (5e-324, 1.0), (float("inf"), 1.0), (2.0 ** 1023, 1.0)):
        fc.fc_add_rn_pos(a, b, ctypes.byref(ok))
        assert ok.value == 0, (a, b)
