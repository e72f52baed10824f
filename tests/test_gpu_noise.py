"""GPU parity of noisy trajectories (qs_run_noisy) and readout error
(qs_readout_error) against the CPU oracle.  Same seed, same draws: the channel
choices agree and the final states agree within 1e-12.  (Damping-type weights
are sums over the state taken in different orders on the two sides; a choice
could only differ for a draw within rounding of a cumulative weight, about
1e-15 per draw, so any disagreement here is a bug.)  Independently, the average
of GPU trajectories converges to the oracle's density matrix."""
import math

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu
TOL = 1e-12
G = w.gate


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available()
    import paper_2212_14201_gb300 as q
    q.build()
    return q


def mixed_rules(n):
    return w.noise_rules([
        w.noise_rule("DEPOLARIZING", None, 0.05),
        w.noise_rule("DAMPING", "CNOT", 0.2),
        w.noise_rule("DECOHERENCE", "H", t1=30.0, t2=20.0, tgate=4.0),
        w.noise_rule("PHASE_DAMPING", "RY", 0.1),
        w.noise_rule("BITFLIP", "X", 0.1),
        w.noise_rule("BITPHASEFLIP", "CZ", 0.15, q0=0, q1=1),
        w.noise_rule("DEPHASING", "T", 0.2),
    ])


def gpu_trajectory(q, n, gates, rules, seed, fuse, rot_err=0.0, params=None, c64=False):
    h = q.qs_alloc_c64(n) if c64 else q.qs_alloc(n)
    try:
        nd = q.qs_run_noisy(h, gates, rules, params=params, rotation_error=rot_err, seed=seed, fuse=fuse)
        return q.qs_get_state(h), nd
    finally:
        q.qs_free(h)


@pytest.mark.parametrize("fuse", [False, True])
@pytest.mark.parametrize("n,ng", [(3, 60), (6, 120), (10, 150)])
def test_trajectories_match_oracle(q, orc, n, ng, fuse):
    rules = mixed_rules(n)
    for seed in range(12):
        g = w.random_circuit(n, ng, 100 + seed)
        rot = 0.03 if seed % 2 else 0.0
        st, nd = orc.run_noisy(n, g, rules, rot_err=rot, seed=seed)
        got, gnd = gpu_trajectory(q, n, g, rules, seed, fuse, rot_err=rot)
        assert gnd == nd, seed
        assert np.max(np.abs(got - orc.as_complex(st))) < TOL, seed


def test_parametrised_gates_and_shared_angles(q, orc):
    n = 5
    g, npar = w.hea_ansatz(n, 3)
    th = w.uniform_angles(npar, 2)
    rules = w.noise_rules([w.noise_rule("DAMPING", "RZ", 0.1), w.noise_rule("DEPOLARIZING", "CNOT", 0.1)])
    for seed in range(6):
        st, nd = orc.run_noisy(n, g, rules, params=th, rot_err=0.02, seed=seed)
        got, gnd = gpu_trajectory(q, n, g, rules, seed, True, rot_err=0.02, params=th)
        assert gnd == nd and np.max(np.abs(got - orc.as_complex(st))) < TOL


def test_average_of_gpu_trajectories_is_the_density_matrix(q, orc):
    n = 3
    g = w.pack([G("H", 0), G("CNOT", 0, 1), G("RX", 2, theta=1.1), G("CZ", 1, 2), G("T", 0), G("H", 2)])
    rules = w.noise_rules([w.noise_rule("DAMPING", "CNOT", 0.2), w.noise_rule("DEPOLARIZING", None, 0.1),
                           w.noise_rule("DECOHERENCE", "H", t1=30.0, t2=20.0, tgate=4.0)])
    rho = orc.dm_run(n, g, rules)
    K = 1500
    acc = np.zeros((8, 8), dtype=np.complex128)
    h = q.qs_alloc(n)
    try:
        for seed in range(K):
            q.qs_set_zero(h)
            q.qs_run_noisy(h, g, rules, seed=10_000 + seed)
            v = q.qs_get_state(h)
            acc += np.outer(v, v.conj())
    finally:
        q.qs_free(h)
    assert np.max(np.abs(acc / K - rho)) < 5 * 0.5 / math.sqrt(K)


def test_unital_noise_fused_equals_per_gate(q):
    n = 18
    g = w.random_circuit(n, 400, 9, two_qubit_prob=0.4)
    rules = w.noise_rules([w.noise_rule("DEPOLARIZING", None, 0.02), w.noise_rule("BITFLIP", "CNOT", 0.05)])
    a, na = gpu_trajectory(q, n, g, rules, 5, True)
    b, nb = gpu_trajectory(q, n, g, rules, 5, False)
    assert na == nb and np.max(np.abs(a - b)) < TOL


def test_complex64_trajectories(q, orc):
    n = 8
    g = w.random_circuit(n, 100, 31)
    rules = mixed_rules(n)
    st, nd = orc.run_noisy(n, g, rules, seed=3)
    got, gnd = gpu_trajectory(q, n, g, rules, 3, True, c64=True)
    assert gnd == nd
    assert np.linalg.norm(got.astype(np.complex128) - orc.as_complex(st)) <= 8 * (len(g) + nd) * 2.0 ** -24


def test_readout_error_matches_oracle(q, orc):
    import torch
    n, shots = 12, 50_000
    rng = np.random.Generator(np.random.PCG64(8))
    samples = rng.integers(0, 1 << n, shots, dtype=np.uint64)
    want = orc.readout(samples, n, 0.9, 0.85, 17)
    host = samples.copy()
    q.qs_readout_error(host, n, 0.9, 0.85, 17)
    assert np.array_equal(host, want)
    dev = torch.tensor(samples.view(np.int64), device="cuda")
    q.qs_readout_error(dev, n, 0.9, 0.85, 17)
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), want)


def test_bad_rules_are_rejected(q):
    h = q.qs_alloc(2)
    try:
        g = w.pack([G("H", 0)])
        for r in (w.noise_rule("DAMPING", None, 1.5), w.noise_rule("DECOHERENCE", None, t1=0.0, t2=1.0, tgate=1.0),
                  (9, -1, -1, -1, 0.1, 0, 0, 0), (0, 99, -1, -1, 0.1, 0, 0, 0)):
            with pytest.raises(q.QsimError):
                q.qs_run_noisy(h, g, w.noise_rules([r]))
    finally:
        q.qs_free(h)


def test_full_size_trajectory(q):
    """n=26 brickwork (depth 20) with depolarizing noise on every gate and damping
    on every CZ: the norm stays 1, the draw count is one per touched qubit and
    rule, and a rerun with the same seed reproduces the state bit for bit."""
    import torch
    n = 26
    g = w.layered_u3_cz(n, 20, 1)
    rules = w.noise_rules([w.noise_rule("DEPOLARIZING", None, 0.01), w.noise_rule("DAMPING", "CZ", 0.01)])
    ncz = int(np.sum(g["type"] == w.GATE_CODES["CZ"]))
    nu3 = len(g) - ncz
    outs = []
    h = q.qs_alloc(n)
    try:
        for _ in range(2):
            q.qs_set_zero(h)
            nd = q.qs_run_noisy(h, g, rules, rotation_error=0.01, seed=77)
            assert nd == nu3 * 2 + ncz * 4   # U3: rotation + depolarizing; CZ: 2 depolarizing + 2 damping
            assert abs(q.qs_probs(h, [])[0] - 1.0) < TOL
            t = torch.empty(2 << n, dtype=torch.float64, device="cuda")
            q.qs_get_state(h, t)
            outs.append(t)
        assert torch.equal(outs[0], outs[1])
    finally:
        q.qs_free(h)
