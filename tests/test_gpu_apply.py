"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on the
same seeded inputs.  Amplitudes within 1e-12 max-abs (complex128); reductions
within 1e-12; samples bit-exact on the same state array."""
import math

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2212_14201_gb300 as q
    q.build()
    return q


@pytest.fixture(params=["fp64", "q60"])
def arith(request, q):
    return {"fp64": q.ARITH_FP64, "q60": q.ARITH_FIXED}[request.param]


def gpu_run(q, n, gates, params=None, plan=None, init=None, arith=None):
    h = q.qs_alloc(n)
    try:
        if arith is not None:
            q.qs_set_arith(h, arith)
        if init is not None:
            q.qs_set_state(h, np.ascontiguousarray(init, dtype=np.complex128))
        q.qs_apply(h, gates, params, plan)
        return q.qs_get_state(h)
    finally:
        q.qs_free(h)


def max_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def test_worked_example_on_gpu(q):
    g = w.pack([w.gate("X", 0), w.gate("Y", 1), w.gate("H", 2), w.gate("RX", 3, theta=math.pi), w.gate("CNOT", 0, 1)])
    psi = gpu_run(q, 4, g)
    want = np.zeros(16, dtype=np.complex128)
    want[9] = want[13] = 1 / math.sqrt(2)
    assert max_err(psi, want) < 1e-15


@pytest.mark.parametrize("name", ["H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "U3", "P"])
def test_every_one_qubit_gate_every_target(q, arith, orc, name):
    n = 9
    init = w.random_state(n, 21)
    for t in range(n):
        for dag in (0, 1):
            g = w.pack([w.gate(name, t, theta=0.3 + t, phi=1.1, lam=-0.7, dagger=dag)])
            ref = orc.as_complex(orc.apply_circuit(init.copy(), n, g))
            got = gpu_run(q, n, g, init=init.view(np.complex128), arith=arith)
            assert max_err(got, ref) < TOL, (name, t, dag)


@pytest.mark.parametrize("name", ["CNOT", "CZ", "CR"])
def test_two_qubit_gates_every_pair(q, arith, orc, name):
    n = 6
    init = w.random_state(n, 22)
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            g = w.pack([w.gate(name, c, t, theta=0.9 + c - t)])
            ref = orc.as_complex(orc.apply_circuit(init.copy(), n, g))
            got = gpu_run(q, n, g, init=init.view(np.complex128), arith=arith)
            assert max_err(got, ref) < TOL, (name, c, t)


def test_multi_controlled_gates(q, arith, orc):
    n = 10
    init = w.random_state(n, 23)
    recs = [w.gate("X", 4, ctrl_mask=0b1000000011), w.gate("U3", 0, theta=1.0, phi=2.0, lam=3.0, ctrl_mask=0b0110000000),
            w.gate("CNOT", 9, 2, ctrl_mask=0b0000110000), w.gate("RZ", 7, theta=0.4, ctrl_mask=0b0000000001),
            w.gate("S", 5, ctrl_mask=0b1111000000, dagger=1), w.gate("Y", 1, ctrl_mask=0b0000001000)]
    g = w.pack(recs)
    ref = orc.as_complex(orc.apply_circuit(init.copy(), n, g))
    assert max_err(gpu_run(q, n, g, init=init.view(np.complex128), arith=arith), ref) < TOL


@pytest.mark.parametrize("n,ng,seed", [(1, 20, 0), (2, 50, 1), (5, 200, 2), (12, 200, 0), (16, 400, 3), (20, 300, 4)])
def test_random_circuits(q, arith, orc, n, ng, seed):
    g = w.random_circuit(n, ng, seed)
    ref = orc.as_complex(orc.run(n, g))
    assert max_err(gpu_run(q, n, g, arith=arith), ref) < TOL


def test_forty_percent_two_qubit_mix(q, arith, orc):
    n = 18
    g = w.random_circuit(n, 500, 2, two_qubit_prob=0.4)
    assert max_err(gpu_run(q, n, g, arith=arith), orc.as_complex(orc.run(n, g))) < TOL


def test_layered_brickwork(q, arith, orc):
    n = 16
    g = w.layered_u3_cz(n, 20, 1)
    assert max_err(gpu_run(q, n, g, arith=arith), orc.as_complex(orc.run(n, g))) < TOL


def test_parametrised_records(q, arith, orc):
    n = 8
    g, npar = w.hea_ansatz(n, 3)
    th = w.uniform_angles(npar, 4)
    assert max_err(gpu_run(q, n, g, params=th, arith=arith), orc.as_complex(orc.run(n, g, th))) < TOL


def test_dagger_roundtrip_identity(q, arith):
    n = 14
    g = w.random_circuit(n, 300, 9)
    both = np.concatenate([g, q.qs_gate_list_dagger(g)])
    psi = gpu_run(q, n, both, arith=arith)
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = 1
    assert max_err(psi, want) < TOL


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_dense_matrix_gate(q, orc, k):
    n = 9
    init = w.random_state(n, 30 + k)
    rng = w.SplitMix64(k)
    targets = []
    while len(targets) < k:
        t = rng.below(n)
        if t not in targets:
            targets.append(t)
    cm = 0
    free = [b for b in range(n) if b not in targets]
    if k < 5:
        cm = 1 << free[-1]
    mat = w.random_matrix(k, 40 + k).view(np.complex128).reshape(1 << k, 1 << k)
    ref = orc.as_complex(orc.apply_matrix(init.copy(), n, targets, mat, cm))
    h = q.qs_alloc(n)
    try:
        q.qs_set_state(h, init.view(np.complex128))
        q.qs_apply_matrix(h, targets, mat, cm)
        got = q.qs_get_state(h)
    finally:
        q.qs_free(h)
    assert max_err(got, ref) < TOL


def test_bad_record_leaves_state_untouched(q):
    n = 4
    h = q.qs_alloc(n)
    try:
        bad = w.pack([w.gate("H", 0), w.gate("X", 7)])
        with pytest.raises(q.QsimError):
            q.qs_apply(h, bad)
        psi = q.qs_get_state(h)
        assert psi[0] == 1 and np.count_nonzero(psi) == 1
    finally:
        q.qs_free(h)


# ---- reductions -------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg0(q, orc):
    """n=12, 200 random gates over the 13 types, seed 0."""
    n = 12
    g = w.random_circuit(n, 200, 0)
    return n, g, orc.run(n, g)


def test_cfg0_probs_and_expect_z(q, orc, cfg0):
    n, g, ref = cfg0
    h = q.qs_alloc(n)
    try:
        q.qs_apply(h, g)
        assert max_err(q.qs_get_state(h), orc.as_complex(ref)) < TOL
        assert max_err(q.qs_probs(h), orc.probs(ref, n)) < TOL
        assert max_err(q.qs_expect_z_all(h), orc.expect_z(ref, n)) < TOL
    finally:
        q.qs_free(h)


@pytest.mark.parametrize("n", [3, 7, 8, 9, 10, 11, 13, 17, 21, 24])
def test_expect_z_sizes(q, orc, n):
    psi = w.random_state_fast(n, n)
    h = q.qs_alloc(n)
    try:
        q.qs_set_state(h, psi.view(np.complex128))
        assert max_err(q.qs_expect_z_all(h), orc.expect_z(psi, n)) < TOL
    finally:
        q.qs_free(h)


@pytest.mark.parametrize("qubits", [[], [0], [5], [3, 1], [11, 0, 6], list(range(12)), [2, 4, 6, 8, 10, 0, 1],
                                    [11, 10, 9, 8, 7, 6, 5, 4, 3, 2, 1, 0], list(range(13)), [12, 0, 5, 7, 3, 9, 1, 2, 4, 6, 8, 10, 11]])
def test_marginals(q, orc, qubits):
    n = 13
    psi = orc.run(n, w.random_circuit(n, 120, 5))
    h = q.qs_alloc(n)
    try:
        q.qs_set_state(h, psi.view(np.complex128))
        assert max_err(q.qs_probs(h, qubits), orc.marginal(psi, n, qubits)) < TOL
    finally:
        q.qs_free(h)


def test_probs_dict(q, orc):
    n = 6
    g = w.pack([w.gate("H", 0), w.gate("CNOT", 0, 3), w.gate("RY", 5, theta=0.3)])
    psi = orc.run(n, g)
    h = q.qs_alloc(n)
    try:
        q.qs_apply(h, g)
        d = q.qs_probs_dict(h, [0, 3, 5], threshold=1e-12)
        m = orc.marginal(psi, n, [0, 3, 5])
        want = {format(k, "03b"): m[k] for k in range(8) if m[k] > 1e-12}
        assert d.keys() == want.keys()
        assert max(abs(d[k] - want[k]) for k in d) < TOL
    finally:
        q.qs_free(h)


@pytest.mark.parametrize("n,nt,seed", [(1, 3, 0), (5, 12, 1), (10, 30, 2), (15, 9, 3)])
def test_pauli_expectations(q, orc, n, nt, seed):
    psi = w.random_state_fast(n, seed)
    psi /= np.linalg.norm(psi)
    terms = w.random_paulis(n, nt, seed + 7)
    h = q.qs_alloc(n)
    try:
        q.qs_set_state(h, psi.view(np.complex128))
        assert abs(q.qs_expect_pauli(h, terms) - orc.expect_pauli(psi, n, terms)) < TOL
        tf = w.tfim(n, 0.7)
        assert abs(q.qs_expect_pauli(h, tf) - orc.expect_pauli(psi, n, tf)) < TOL
    finally:
        q.qs_free(h)


def _pauli_structure_terms(n):
    """Terms that exercise every pass layout: the identity, Z strings beyond one
    pass, one X mask shared by more terms than a pass holds, X masks with equal
    leading bits and their sum, and Y counts of every residue mod 4."""
    rows = [(0.3, 0, 0)]
    rows += [(0.01 * (k + 1), 0, (k * 37 + 5) % (1 << n)) for k in range(15)]
    shared = 0b101001 & ((1 << n) - 1)
    rows += [(0.02 * (k - 9), shared, (k * 11) % (1 << n)) for k in range(17)]
    full = (1 << n) - 1
    a, b = ((1 << (n - 1)) | 0b110) & full, ((1 << (n - 1)) | 0b011) & full
    rows += [(0.4, a, 0), (-0.25, b, 1 << (n - 1)), (0.15, a ^ b, 0b101 & full)]
    for ny in range(4):  # Y on qubits 0..ny-1, X on the top two
        ys = ((1 << ny) - 1) & full
        rows.append((0.1 * (ny + 1), ys | (0b11 << (n - 2)), ys))
    rows.append((-0.2, full, full))  # Y on every qubit
    rows.append((0.05, full, 0))     # X on every qubit
    return np.array(rows, dtype=w.PAULI_DTYPE)


@pytest.mark.parametrize("n", [2, 9, 14])
def test_pauli_pass_layouts(q, orc, n):
    psi = w.random_state_fast(n, 40 + n)
    psi /= np.linalg.norm(psi)
    terms = _pauli_structure_terms(n)
    h = q.qs_alloc(n)
    try:
        q.qs_set_state(h, psi.view(np.complex128))
        assert abs(q.qs_expect_pauli(h, terms) - orc.expect_pauli(psi, n, terms)) < TOL
        for t in terms:  # each term on its own
            one = np.array([t], dtype=w.PAULI_DTYPE)
            assert abs(q.qs_expect_pauli(h, one) - orc.expect_pauli(psi, n, one)) < TOL
    finally:
        q.qs_free(h)


def test_pauli_large_state_and_fp64_fallback(q, orc):
    """n=22 (several CTAs per pass, every cell basis) and a state of norm^2 = 2,
    outside the fixed-point bound, which takes the FP64 kernel."""
    n = 22
    psi = w.random_state_fast(n, 9)
    psi /= np.linalg.norm(psi)
    terms = np.concatenate([w.tfim(n, 0.7), w.random_paulis(n, 25, 3)])
    h = q.qs_alloc(n)
    try:
        q.qs_set_state(h, psi.view(np.complex128))
        want = orc.expect_pauli(psi, n, terms)
        got = q.qs_expect_pauli(h, terms)
        assert abs(got - want) < TOL
        assert q.qs_expect_pauli(h, terms) == got  # integer sums: identical on every call
        big = psi * np.sqrt(2.0)
        q.qs_set_state(h, big.view(np.complex128))
        assert abs(q.qs_expect_pauli(h, terms) - 2.0 * want) < 4 * TOL
    finally:
        q.qs_free(h)


# ---- sampler: bit-exact on the same state array -----------------------------------------

@pytest.mark.parametrize("n,seed", [(1, 1), (4, 2), (10, 3), (12, 0), (15, 5), (20, 6), (21, 7), (24, 8)])
def test_sampler_bit_exact(q, orc, n, seed):
    g = w.random_circuit(n, 100, seed)
    h = q.qs_alloc(n)
    try:
        q.qs_apply(h, g)
        st = q.qs_get_state(h).view(np.float64).copy()
        got = q.qs_sample(h, 11 + seed, 20000)
        assert np.array_equal(got, orc.sample(st, n, 11 + seed, 20000))
    finally:
        q.qs_free(h)


def _canonical_cdf(orc, st, n):
    """The canonical sampler's decision values on a state array (interleaved f64):
    E[b] (block prefixes, from the oracle) and C_x = E[b] + left-to-right partial
    sum of p within x's block (numpy's accumulate is sequential, p = re*re + im*im
    with separate roundings, as in the oracle)."""
    E = orc.block_prefix(st, n)
    re, im = st[0::2], st[1::2]
    p = re * re + im * im
    L = min(1024, 1 << n)
    S = np.add.accumulate(p.reshape(-1, L), axis=1)
    return E, (E[:-1, None] + S).reshape(-1)


@pytest.mark.parametrize("n,seed,fused", [(12, 0, False), (20, 6, True)])
def test_sampler_cross_state_explained_flips(q, orc, n, seed, fused):
    """Samples of the GPU-computed state against samples of the oracle-computed
    state (the same program, computed independently on both sides): a shot may
    differ only where its draw u_s lies between the two sides' decision values at
    a boundary between the two picks (min(C_x, C'_x) <= u_s < max(C_x, C'_x), or
    the same for a block prefix).  Any other mismatch fails."""
    g = w.random_circuit(n, 200, seed)
    shots, sseed = 1_000_000, 31 + seed
    ref = orc.run(n, g)
    plan = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5) if fused else None
    h = q.qs_alloc(n)
    try:
        q.qs_apply(h, g, None, plan)
        got = q.qs_sample(h, sseed, shots)
        st = q.qs_get_state(h).view(np.float64).copy()
    finally:
        q.qs_free(h)
        if plan is not None:
            q.qs_plan_free(plan)
    # the definition on the GPU's own state: bit-exact
    assert np.array_equal(got, orc.sample(st, n, sseed, shots))
    want = orc.sample(ref, n, sseed, shots)
    bad = np.nonzero(got != want)[0]
    if bad.size:
        Eg, Cg = _canonical_cdf(orc, st, n)
        Eo, Co = _canonical_cdf(orc, ref, n)
        L = min(1024, 1 << n)
        for s in bad:
            u = (orc.splitmix64(sseed, int(s)) >> 11) * 2.0 ** -53
            lo, hi = sorted((int(got[s]), int(want[s])))
            xs = np.arange(lo, hi + 1)
            straddle = np.any((np.minimum(Cg[xs], Co[xs]) <= u) & (u < np.maximum(Cg[xs], Co[xs])))
            bs = np.arange(lo // L, hi // L + 1)
            straddle |= bool(np.any((np.minimum(Eg[bs + 1], Eo[bs + 1]) <= u) & (u < np.maximum(Eg[bs + 1], Eo[bs + 1]))))
            assert straddle, f"shot {s}: GPU {got[s]} oracle {want[s]} not explained by the two states' rounding"
    print(f"n={n}: {bad.size} explained flips in {shots} shots")


def test_sampler_edge_states(q, orc):
    n = 5
    for amps in [np.zeros(1 << n, dtype=np.complex128), None]:
        h = q.qs_alloc(n)
        try:
            if amps is None:
                amps = np.zeros(1 << n, dtype=np.complex128)
                amps[3] = 0.5   # total probability 0.25 -> most draws fall back
                amps[17] = 0.25j
            q.qs_set_state(h, amps)
            got = q.qs_sample(h, 5, 3000)
            assert np.array_equal(got, orc.sample(amps.view(np.float64), n, 5, 3000))
        finally:
            q.qs_free(h)


def test_sampler_device_output(q, orc):
    import torch
    n = 11
    g = w.random_circuit(n, 80, 3)
    h = q.qs_alloc(n)
    try:
        q.qs_apply(h, g)
        out = torch.empty(5000, dtype=torch.int64, device="cuda")
        q.qs_sample(h, 99, 5000, out)
        q.qs_sync(h)
        st = q.qs_get_state(h).view(np.float64).copy()
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), orc.sample(st, n, 99, 5000))
    finally:
        q.qs_free(h)


def test_statevector_class_on_torch_memory(q, orc):
    import torch
    n = 10
    g = w.random_circuit(n, 100, 8)
    sv = q.StateVector(n)
    sv.apply(g)
    ref = orc.run(n, g)
    assert max_err(sv.state(), orc.as_complex(ref)) < TOL
    t = sv.amps.view(torch.complex128).cpu().numpy()
    assert max_err(t, orc.as_complex(ref)) < TOL
    sv.close()


def test_arith_modes_and_bound_tracking(q, orc):
    n = 10
    g = w.random_circuit(n, 150, 12)
    ref = orc.as_complex(orc.run(n, g))
    big = np.zeros(1 << n, dtype=np.complex128)
    big[5] = 3.0   # norm 3: beyond the Q60 range
    h = q.qs_alloc(n)
    try:
        for mode in (q.ARITH_AUTO, q.ARITH_FP64, q.ARITH_FIXED):
            q.qs_set_arith(h, mode)
            q.qs_set_zero(h)
            q.qs_apply(h, g)
            assert max_err(q.qs_get_state(h), ref) < TOL
        q.qs_set_state(h, big)
        q.qs_set_arith(h, q.ARITH_FIXED)
        with pytest.raises(q.QsimError):
            q.qs_apply(h, g)
        q.qs_set_arith(h, q.ARITH_AUTO)   # falls back to FP64 for the large state
        q.qs_apply(h, g)
        want = orc.as_complex(orc.apply_circuit(big.copy().view(np.float64), n, g))
        assert max_err(q.qs_get_state(h), want) < 4 * TOL
    finally:
        q.qs_free(h)


def test_exact_marginals_match_fp64_and_oracle(q, orc):
    """A state reached from |0> by gates has known-bounded components, so its
    squared norm and marginals over <= 3 qubits are summed exactly in integers;
    a state loaded with qs_set_state takes the FP64 kernels.  Both agree with the
    oracle on the same amplitudes (1e-13), and a zero branch is exactly zero."""
    n = 14
    g = w.random_circuit(n, 200, 9)
    h = q.qs_alloc(n)
    h2 = q.qs_alloc(n)
    try:
        q.qs_apply(h, g)
        st = q.qs_get_state(h)
        q.qs_set_state(h2, st)
        ref_st = st.view(np.float64)
        for qs_ in ([], [0], [13], [3, 7], [1, 5, 12]):
            exact = q.qs_probs(h, qs_)
            fp64 = q.qs_probs(h2, qs_)
            ref = orc.marginal(ref_st, n, qs_)
            assert np.max(np.abs(exact - ref)) < 1e-13, qs_
            assert np.max(np.abs(fp64 - ref)) < 1e-13, qs_
        q.qs_set_zero(h)
        p = q.qs_probs(h, [4, 9])
        assert p[0] == 1.0 and np.all(p[1:] == 0.0)
    finally:
        q.qs_free(h)
        q.qs_free(h2)


def test_sampler_bit_exact_n31(q, orc):
    """n=31: 2048 superblocks of 1024 blocks, so the prefix of the superblock
    totals runs in chunks; 20000 shots against the oracle on the same 32 GiB of
    amplitudes (skipped without room for the host copy)."""
    import os
    import torch
    n = 31
    need = (16 << n) * 2.2
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 0
    free_dev, _ = torch.cuda.mem_get_info()
    if avail < need or free_dev < (16 << n) * 1.1:
        pytest.skip("not enough host or device memory for a 32 GiB state and its copy")
    g = w.random_circuit(n, 60, 31)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    h = q.qs_alloc(n)
    try:
        q.qs_apply(h, g, None, p)
        got = q.qs_sample(h, 77, 20000)
        st = q.qs_get_state(h).view(np.float64)
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)
    assert np.array_equal(got, orc.sample(st, n, 77, 20000))
