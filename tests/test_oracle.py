"""Pins for the CPU oracle: each check compares it with something other than itself
(worked examples of the paper, closed forms, textbook identities, library routines,
brute force on small inputs), chosen so that a dropped term, a wrong sign or index or
a transposed operand in the oracle fails at least one of them."""
import math
import os

import numpy as np
import pytest

import workloads as w

GOLD = os.path.join(os.path.dirname(__file__), "golden")
R2 = 1.0 / math.sqrt(2.0)


def cvec(s):
    return s.view(np.complex128)


# --- worked examples from the paper's listings --------------------------------------

def test_fusion_listing_example(orc):
    g = w.pack([w.gate("X", 0), w.gate("Y", 1), w.gate("H", 2), w.gate("RX", 3, theta=math.pi),
                w.gate("CNOT", 0, 1)])
    psi = cvec(orc.run(4, g))
    want = np.zeros(16, dtype=np.complex128)
    for line in open(os.path.join(GOLD, "fusion_listing_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        i, re, im = line.split()
        want[int(i)] = complex(float(re), float(im))
    assert np.max(np.abs(psi - want)) < 1e-15


def test_qif_branches(orc):
    rows = [l.split() for l in open(os.path.join(GOLD, "qif_branches.txt")) if l.strip() and not l.startswith("#")]
    false = cvec(orc.run(3, w.pack([w.gate("H", 0), w.gate("CNOT", 0, 1), w.gate("CNOT", 1, 2)])))
    true = cvec(orc.run(3, w.pack([w.gate("H", 0), w.gate("H", 1), w.gate("H", 2)])))
    want_f = np.zeros(8, dtype=np.complex128)
    for br, idx, re, im in rows:
        if br == "false":
            want_f[int(idx)] = complex(float(re), float(im))
        else:
            want_t = np.full(8, complex(float(re), float(im)))
    assert np.max(np.abs(false - want_f)) < 1e-15
    assert np.max(np.abs(true - want_t)) < 1e-15


# --- closed forms ---------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 10])
def test_ghz(orc, n):
    recs = [w.gate("H", 0)] + [w.gate("CNOT", q, q + 1) for q in range(n - 1)]
    psi = cvec(orc.run(n, w.pack(recs)))
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = want[-1] = R2
    assert np.max(np.abs(psi - want)) < 1e-15


def qft_records(n):
    """QFT for the little-endian index: H and controlled phases from the top qubit
    down, then the qubit reversal with three CNOTs per swap."""
    recs = []
    for q in range(n - 1, -1, -1):
        recs.append(w.gate("H", q))
        for r in range(q - 1, -1, -1):
            recs.append(w.gate("CR", r, q, theta=math.pi / (1 << (q - r))))
    for q in range(n // 2):
        a, b = q, n - 1 - q
        recs += [w.gate("CNOT", a, b), w.gate("CNOT", b, a), w.gate("CNOT", a, b)]
    return recs


@pytest.mark.parametrize("n,j", [(1, 1), (3, 5), (6, 37), (9, 300)])
def test_qft_basis_state_matches_numpy_fft(orc, n, j):
    prep = [w.gate("X", q) for q in range(n) if (j >> q) & 1]
    psi = cvec(orc.run(n, w.pack(prep + qft_records(n))))
    e = np.zeros(1 << n, dtype=np.complex128)
    e[j] = 1.0
    want = np.fft.ifft(e) * math.sqrt(1 << n)   # e^{2 pi i j k / N} / sqrt(N)
    assert np.max(np.abs(psi - want)) < 1e-13


def test_single_qubit_columns_closed_form(orc):
    th, ph, la = 0.7, 1.9, -2.3
    cases = {
        "RX": [math.cos(th / 2), -1j * math.sin(th / 2)],
        "RY": [math.cos(th / 2), math.sin(th / 2)],
        "RZ": [np.exp(-0.5j * th), 0],
        "U3": [math.cos(th / 2), np.exp(1j * ph) * math.sin(th / 2)],
        "H": [R2, R2], "X": [0, 1], "Y": [0, 1j], "Z": [1, 0],
    }
    for name, col in cases.items():
        psi = cvec(orc.run(1, w.pack([w.gate(name, 0, theta=th, phi=ph, lam=la)])))
        assert np.max(np.abs(psi - np.array(col))) < 1e-15, name
    # second column via X first: |1> input
    cols1 = {
        "S": [0, 1j], "T": [0, np.exp(0.25j * math.pi)], "P": [0, np.exp(1j * th)],
        "U3": [-np.exp(1j * la) * math.sin(th / 2), np.exp(1j * (ph + la)) * math.cos(th / 2)],
        "RZ": [0, np.exp(0.5j * th)], "Y": [-1j, 0], "Z": [0, -1], "H": [R2, -R2],
    }
    for name, col in cols1.items():
        psi = cvec(orc.run(1, w.pack([w.gate("X", 0), w.gate(name, 0, theta=th, phi=ph, lam=la)])))
        assert np.max(np.abs(psi - np.array(col))) < 1e-15, name


# --- textbook identities between gates (pin the matrices against each other) ----------

def _apply(orc, n, state, recs):
    return cvec(orc.apply_circuit(state.copy().view(np.float64), n, w.pack(recs)))


def test_gate_identities(orc):
    n = 3
    psi0 = cvec(w.random_state(n, 5))
    th, ph = 1.234, -0.77
    same = [
        ([w.gate("H", 1), w.gate("X", 1), w.gate("H", 1)], [w.gate("Z", 1)]),
        ([w.gate("S", 0), w.gate("S", 0)], [w.gate("Z", 0)]),
        ([w.gate("T", 2), w.gate("T", 2)], [w.gate("S", 2)]),
        ([w.gate("U3", 1, theta=th, phi=-math.pi / 2, lam=math.pi / 2)], [w.gate("RX", 1, theta=th)]),
        ([w.gate("U3", 1, theta=th, phi=0.0, lam=0.0)], [w.gate("RY", 1, theta=th)]),
        ([w.gate("H", 0), w.gate("RZ", 0, theta=th), w.gate("H", 0)], [w.gate("RX", 0, theta=th)]),
        ([w.gate("H", 1), w.gate("CZ", 0, 1), w.gate("H", 1)], [w.gate("CNOT", 0, 1)]),
        ([w.gate("CR", 2, 0, theta=math.pi)], [w.gate("CZ", 0, 2)]),
        ([w.gate("RZ", 2, theta=th), w.gate("RZ", 2, theta=ph)], [w.gate("RZ", 2, theta=th + ph)]),
        ([w.gate("RY", 0, theta=th, dagger=1)], [w.gate("RY", 0, theta=-th)]),
        ([w.gate("U3", 0, theta=th, phi=ph, lam=0.4, dagger=1)], [w.gate("U3", 0, theta=-th, phi=-0.4, lam=-ph)]),
        ([w.gate("X", 0, ctrl_mask=0b110)], [w.gate("CNOT", 1, 0, ctrl_mask=0b100)]),
    ]
    for a, b in same:
        assert np.max(np.abs(_apply(orc, n, psi0, a) - _apply(orc, n, psi0, b))) < 1e-14, (a, b)
    # Y = i X Z ; RZ(th) = e^{-i th/2} P(th)
    y = _apply(orc, n, psi0, [w.gate("Y", 1)])
    xz = _apply(orc, n, psi0, [w.gate("Z", 1), w.gate("X", 1)])
    assert np.max(np.abs(y - 1j * xz)) < 1e-15
    rz = _apply(orc, n, psi0, [w.gate("RZ", 2, theta=th)])
    p = _apply(orc, n, psi0, [w.gate("P", 2, theta=th)])
    assert np.max(np.abs(rz - np.exp(-0.5j * th) * p)) < 1e-15


# --- brute force: full 2^n x 2^n operators built with np.kron -------------------------

def full_operator(orc, n, rec):
    """Dense operator of one record: sum over control projector P1(C) x U_t + (I - P1(C)) x I."""
    t, cm, u = orc.gate_matrix(np.array([rec], dtype=w.GATE_DTYPE)[0:1], n)
    I2 = np.eye(2)
    P1 = np.diag([0.0, 1.0])
    on = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):  # kron puts the leftmost factor on the most significant bit
        if q == t:
            f = u
        elif (cm >> q) & 1:
            f = P1
        else:
            f = I2
        on = np.kron(on, f)
    proj = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        proj = np.kron(proj, P1 if (cm >> q) & 1 else I2)
    return on + (np.eye(1 << n) - proj)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (4, 2), (6, 3), (8, 4)])
def test_circuit_matches_kron_product(orc, n, seed):
    g = w.random_circuit(n, 40, seed)
    psi = cvec(orc.run(n, g))
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = 1
    for rec in g:
        ref = full_operator(orc, n, rec) @ ref
    assert np.max(np.abs(psi - ref)) < 1e-13


def test_multicontrol_matches_kron(orc):
    n = 5
    psi0 = cvec(w.random_state(n, 9))
    recs = [w.gate("U3", 2, theta=0.3, phi=1.1, lam=-0.4, ctrl_mask=0b10011),
            w.gate("CNOT", 4, 0, ctrl_mask=0b01000), w.gate("RY", 1, theta=2.2, ctrl_mask=0b00100, dagger=1)]
    got = _apply(orc, n, psi0, recs)
    ref = psi0.copy()
    for r in recs:
        ref = full_operator(orc, n, np.array([r], dtype=w.GATE_DTYPE)[0]) @ ref
    assert np.max(np.abs(got - ref)) < 1e-14


def test_dense_matrix_gate_matches_kron(orc):
    n = 6
    psi0 = cvec(w.random_state(n, 3))
    for k, targets, cm in [(1, [4], 0), (2, [5, 1], 0b000100), (3, [0, 3, 2], 0b100000), (5, [1, 5, 0, 4, 2], 0)]:
        m = w.random_matrix(k, 17 + k).view(np.complex128).reshape(1 << k, 1 << k)
        got = cvec(orc.apply_matrix(psi0.copy().view(np.float64), n, targets, m, cm))
        # permute qubits so the targets become the k lowest bits (target j -> bit j), apply I x M
        order = list(targets) + [q for q in range(n) if q not in targets]
        t = psi0.reshape([2] * n)  # axis a is qubit n-1-a
        axes = [n - 1 - q for q in reversed(order)]
        tt = np.transpose(t, axes).reshape(-1)
        # after transposition bit j of the new index is qubit order[j]
        rest = n - k
        blocks = tt.reshape(1 << rest, 1 << k)
        cm_rest = sum(1 << i for i, q in enumerate(order[k:]) if (cm >> q) & 1)
        newb = blocks.copy()
        for r in range(1 << rest):
            if (r & cm_rest) == cm_rest:
                newb[r] = m @ blocks[r]
        back = np.transpose(newb.reshape([2] * n), np.argsort(axes)).reshape(-1)
        assert np.max(np.abs(got - back)) < 1e-14, k


# --- invariants ------------------------------------------------------------------------

@pytest.mark.parametrize("n,seed", [(3, 0), (7, 1), (12, 2)])
def test_norm_and_dagger_roundtrip(orc, n, seed):
    g = w.random_circuit(n, 200, seed)
    psi = orc.run(n, g)
    assert abs(np.linalg.norm(cvec(psi)) - 1.0) < 1e-12
    inv = g[::-1].copy()
    inv["dagger"] = 1 - inv["dagger"]
    back = cvec(orc.apply_circuit(psi, n, inv))
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = 1
    assert np.max(np.abs(back - want)) < 1e-12


# --- reductions --------------------------------------------------------------------------

def test_product_state_expectations(orc):
    n = 4
    ths = [0.3, 1.7, 2.9, 4.4]
    phs = [0.1, -1.2, 2.0, 0.9]
    recs = [w.gate("U3", q, theta=ths[q], phi=phs[q], lam=0.5 * q) for q in range(n)]
    psi = orc.run(n, w.pack(recs))
    ez = orc.expect_z(psi, n)
    assert np.max(np.abs(ez - np.cos(ths))) < 1e-14
    for q in range(n):
        ex = orc.expect_pauli(psi, n, np.array([(1.0, 1 << q, 0)], dtype=w.PAULI_DTYPE))
        ey = orc.expect_pauli(psi, n, np.array([(1.0, 1 << q, 1 << q)], dtype=w.PAULI_DTYPE))
        assert abs(ex - math.sin(ths[q]) * math.cos(phs[q])) < 1e-14
        assert abs(ey - math.sin(ths[q]) * math.sin(phs[q])) < 1e-14
    zz = orc.expect_pauli(psi, n, w.zz_chain(n))
    assert abs(zz - sum(math.cos(ths[i]) * math.cos(ths[i + 1]) for i in range(n - 1))) < 1e-14


def test_cz_layer_keeps_z(orc):
    # one brickwork layer: U3 then CZs; CZ commutes with Z so <Z_i> = cos(theta_i)
    n = 8
    g = w.layered_u3_cz(n, 1, 1)
    psi = orc.run(n, g)
    assert np.max(np.abs(orc.expect_z(psi, n) - np.cos(g["p"][:n, 0]))) < 1e-14


_PAULI = {0: np.eye(2), 1: np.array([[0, 1], [1, 0]]), 2: np.array([[0, -1j], [1j, 0]]), 3: np.diag([1.0, -1.0])}


def pauli_matrix(n, xm, zm):
    m = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        k = ((xm >> q) & 1) + 2 * ((zm >> q) & 1)   # 0 I, 1 X, 2 Z, 3 Y
        m = np.kron(m, _PAULI[{0: 0, 1: 1, 2: 3, 3: 2}[k]])
    return m


def test_pauli_sum_matches_dense(orc):
    n = 5
    psi = w.random_state(n, 11)
    terms = w.random_paulis(n, 12, 4)
    H = sum(t["coef"] * pauli_matrix(n, int(t["xmask"]), int(t["zmask"])) for t in terms)
    v = cvec(psi)
    assert abs(orc.expect_pauli(psi, n, terms) - np.vdot(v, H @ v).real) < 1e-13
    assert np.max(np.abs(cvec(orc.apply_pauli_sum(psi, n, terms)) - H @ v)) < 1e-14


def test_marginal_and_probs(orc):
    n = 7
    psi = orc.run(n, w.random_circuit(n, 60, 8))
    p = orc.probs(psi, n)
    v = cvec(psi)
    assert np.array_equal(p, v.real * v.real + v.imag * v.imag)
    assert abs(p.sum() - 1) < 1e-13
    q = [5, 0, 3]
    m = orc.marginal(psi, n, q)
    t = p.reshape([2] * n)  # axis a <-> qubit n-1-a
    keep = [n - 1 - x for x in q]
    ref = t.sum(axis=tuple(a for a in range(n) if a not in keep))
    # remaining axes are in increasing axis order; reorder so bit j = qubit q[j]
    rem = sorted(keep)
    ref = np.transpose(ref, [rem.index(n - 1 - x) for x in reversed(q)]).reshape(-1)
    assert np.max(np.abs(m - ref)) < 1e-15
    ez = orc.expect_z(psi, n)
    for i in range(n):
        assert abs(ez[i] - orc.marginal(psi, n, [i]) @ np.array([1.0, -1.0])) < 1e-14


# --- sampler ---------------------------------------------------------------------------

def test_splitmix64_published_vector(orc):
    # SplitMix64 seeded with 0: first outputs of the reference generator
    # (Steele, Lea & Flood 2014; Vigna's splitmix64.c).
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert orc.splitmix64(0, 2) == 0x06C45D188009454F


def _brute_sample(psi_f, n, seed, shots, orc):
    """Smallest x with C_x > u, C built element by element in the canonical order."""
    v = cvec(psi_f)
    N = 1 << n
    L = min(1024, N)
    p = [float(a.real) * float(a.real) + float(a.imag) * float(a.imag) for a in v]
    C = []
    E = 0.0
    for b in range(N // L):
        S = 0.0
        for j in range(L):
            S += p[b * L + j]
            C.append(E + S)
        E = E + S
    out = []
    last = max(i for i in range(N) if p[i] > 0)
    for s in range(shots):
        u = (orc.splitmix64(seed, s) >> 11) * 2.0 ** -53
        x = next((i for i in range(N) if C[i] > u), None)
        out.append(last if x is None else x)
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("n,seed", [(1, 3), (4, 5), (11, 7), (12, 8)])
def test_sampler_matches_brute_force(orc, n, seed):
    psi = orc.run(n, w.random_circuit(n, 50, seed))
    got = orc.sample(psi, n, 99 + seed, 300)
    assert np.array_equal(got, _brute_sample(psi, n, 99 + seed, 300, orc))


def test_sampler_norm_deficit_and_point_mass(orc):
    n = 3
    psi = orc.run(n, w.pack([w.gate("X", 1)]))
    assert set(orc.sample(psi, n, 1, 500).tolist()) == {2}
    # total probability 0.25: draws above the total fall back to the last x with p_x > 0
    half = orc.run(n, w.pack([w.gate("H", 0), w.gate("H", 2)])) * 0.5
    got = orc.sample(half, n, 4, 400)
    assert np.array_equal(got, _brute_sample(half, n, 4, 400, orc))
    assert (got == 5).sum() > 200


def _two_level_cumulative(psi_f, n):
    """C_x of the canonical sampler built with numpy's cumulative sums, which add
    left to right: block sums, then per-superblock prefixes of the block totals,
    offset by the prefix of the superblock totals."""
    v = cvec(psi_f)
    p = v.real * v.real + v.imag * v.imag
    N = 1 << n
    L = min(1024, N)
    nb = N // L
    G = min(1024, nb)
    S = np.cumsum(p.reshape(nb, L), axis=1)          # S_b(j)
    T = S[:, -1]
    F = np.cumsum(T.reshape(nb // G, G), axis=1)     # F_c(i)
    P = np.concatenate([[0.0], np.cumsum(F[:, -1])])[:-1]
    Eend = (P[:, None] + F).reshape(nb)              # E_{b+1}
    E = np.concatenate([[0.0], Eend])
    C = E[:-1, None] + S                             # E_b + S_b(x - bL)
    return E, C.reshape(N), p


def test_sampler_superblocks(orc):
    """n=21: two superblocks of 1024 blocks.  The oracle's block prefixes equal the
    definition rebuilt from numpy's left-to-right cumulative sums; they never
    decrease, end at the exact total within the summation bound, and every shot is
    the first x with C_x above its draw."""
    n = 21
    psi = w.random_state_fast(n, 5)   # generic values: the two-level sums round differently
    psi /= math.sqrt(math.fsum((psi * psi).tolist()))
    E = orc.block_prefix(psi, n)
    E2, C, p = _two_level_cumulative(psi, n)
    assert np.array_equal(E, E2)
    one_level = np.concatenate([[0.0], np.cumsum(np.cumsum(p.reshape(-1, 1024), axis=1)[:, -1])])
    assert not np.array_equal(E, one_level)   # the case distinguishes the two definitions
    assert E[0] == 0.0 and np.all(np.diff(E) >= 0.0)
    total = math.fsum(p.tolist())
    assert abs(E[-1] - total) <= (1024 + 1024 + 2 + 2) * 2.0 ** -53 * total
    # the second superblock starts from the first one's total: its first prefix is
    # that total plus the next block total, rounded once
    T1024 = float(np.cumsum(p[1024 * 1024:1025 * 1024])[-1])
    assert E[1025] == E[1024] + T1024
    seed, shots = 17, 2000
    got = orc.sample(psi, n, seed, shots)
    u = np.array([(orc.splitmix64(seed, s) >> 11) * 2.0 ** -53 for s in range(shots)])
    want = np.searchsorted(C, u, side="right")
    last = int(np.nonzero(p > 0)[0].max())
    want = np.where(want >= len(C), last, want).astype(np.uint64)
    assert np.array_equal(got, want)
    # both superblocks are drawn in proportion to their mass
    hi = float(p[1 << 20:].sum())
    frac = float(np.mean(got >= (1 << 20)))
    assert abs(frac - hi) < 5 * math.sqrt(hi * (1 - hi) / shots)


def test_sampler_chi_square(orc):
    from scipy.stats import chisquare
    n = 12
    psi = orc.run(n, w.random_circuit(n, 200, 0))
    shots = 1_000_000
    s = orc.sample(psi, n, 11, shots)
    p = orc.probs(psi, n)
    counts = np.bincount(s.astype(np.int64), minlength=1 << n)
    keep = p * shots >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(p[keep], p[~keep].sum()) * shots
    exp *= obs.sum() / exp.sum()
    assert chisquare(obs, exp).pvalue > 1e-4


# --- adjoint gradient --------------------------------------------------------------------

@pytest.mark.parametrize("n,layers", [(2, 2), (4, 3), (6, 2)])
def test_adjoint_matches_parameter_shift(orc, n, layers):
    g, npar = w.hea_ansatz(n, layers)
    th = w.uniform_angles(npar, 4)
    H = w.tfim(n, 0.7)
    e, grad = orc.adjoint_grad(n, g, th, H)
    assert abs(e - orc.energy(n, g, th, H)) < 1e-13
    shift = np.empty(npar)
    for k in range(npar):
        tp, tm = th.copy(), th.copy()
        tp[k] += math.pi / 2
        tm[k] -= math.pi / 2
        shift[k] = 0.5 * (orc.energy(n, g, tp, H) - orc.energy(n, g, tm, H))
    assert np.max(np.abs(grad - shift)) <= 1e-9 * max(1.0, np.max(np.abs(shift)))


def test_adjoint_matches_finite_differences_with_controls_and_dagger(orc):
    n = 4
    recs = [w.gate("H", q) for q in range(n)]
    recs += [w.gate("RX", 1, param_idx=0, ctrl_mask=0b0001), w.gate("CR", 2, 3, param_idx=1),
             w.gate("RY", 0, param_idx=2, dagger=1), w.gate("P", 2, param_idx=0),
             w.gate("RZ", 3, param_idx=3), w.gate("CNOT", 3, 1), w.gate("RX", 2, param_idx=2)]
    g = w.pack(recs)
    th = np.array([0.4, 1.3, -0.8, 2.2])
    H = w.random_paulis(n, 6, 2)
    e, grad = orc.adjoint_grad(n, g, th, H)
    h = 1e-6
    fd = np.empty(4)
    for k in range(4):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (orc.energy(n, g, tp, H) - orc.energy(n, g, tm, H)) / (2 * h)
    assert np.max(np.abs(grad - fd)) < 1e-7


def test_oracle_rejects_bad_records(orc):
    with pytest.raises(orc.OracleError):
        orc.run(3, w.pack([w.gate("H", 3)]))
    with pytest.raises(orc.OracleError):
        orc.run(3, w.pack([w.gate("CNOT", 1, 1)]))
    with pytest.raises(orc.OracleError):
        orc.run(3, w.pack([w.gate("X", 0, ctrl_mask=0b1)]))
