"""Pins of the oracle's noise channels, trajectories and readout error (the
paper's NoiseQVM: Kraus operator models, set_readout_error, set_rotation_error)
against channel algebra and closed forms: completeness, the effect of each
channel on |0>, |1>, |+> (T1 population decay and T2 coherence decay for the
decoherence model), the trajectory average against the density-matrix
evolution, and the draw definitions."""
import math

import numpy as np
import pytest

import workloads as w

G = w.gate
M = w.NOISE_MODELS


def u01(orc, seed, k):
    return (orc.splitmix64(seed, k) >> 11) * 2.0 ** -53


@pytest.mark.parametrize("model", list(M))
def test_kraus_sets_are_complete(orc, model):
    for p in (0.0, 0.03, 0.5, 1.0):
        K, unital = orc.kraus(M[model], p, 40.0, 25.0, 3.0)
        S = sum(k.conj().T @ k for k in K)
        assert np.max(np.abs(S - np.eye(2))) < 1e-15
        if unital:     # every operator a scaled unitary
            for k in K:
                c2 = float(np.real(np.trace(k.conj().T @ k))) / 2
                assert np.max(np.abs(k.conj().T @ k - c2 * np.eye(2))) < 1e-15


def one_gate_dm(orc, prep, model, p, **kw):
    """Density matrix after `prep` (gates on one qubit) followed by the channel
    (attached to an identity gate)."""
    gates = w.pack(prep + [G("I", 0)])
    rules = w.noise_rules([w.noise_rule(model, "I", p, **kw)])
    return orc.dm_run(1, gates, rules)


def test_channel_closed_forms(orc):
    p = 0.23
    X, H = [G("X", 0)], [G("H", 0)]
    assert abs(one_gate_dm(orc, X, "DAMPING", p)[1, 1] - (1 - p)) < 1e-15
    assert abs(one_gate_dm(orc, X, "DAMPING", p)[0, 0] - p) < 1e-15
    r = one_gate_dm(orc, H, "PHASE_DAMPING", p)
    assert abs(r[0, 1] - math.sqrt(1 - p) / 2) < 1e-15 and abs(r[0, 0] - 0.5) < 1e-15
    for m in ("DEPHASING", "PHASEFLIP"):
        assert abs(one_gate_dm(orc, H, m, p)[0, 1] - (1 - 2 * p) / 2) < 1e-15
    assert abs(one_gate_dm(orc, [], "BITFLIP", p)[1, 1] - p) < 1e-15
    assert abs(one_gate_dm(orc, [], "BITPHASEFLIP", p)[1, 1] - p) < 1e-15
    assert abs(one_gate_dm(orc, H, "BITPHASEFLIP", p)[0, 1] - (1 - 2 * p) / 2) < 1e-15
    # depolarizing: rho -> (1 - p) rho + p I / 2
    assert abs(one_gate_dm(orc, [], "DEPOLARIZING", p)[0, 0] - (1 - p / 2)) < 1e-15
    assert abs(one_gate_dm(orc, H, "DEPOLARIZING", p)[0, 1] - (1 - p) / 2) < 1e-15
    # decoherence: population decays with T1, coherence with T2
    t1, t2, tg = 40.0, 25.0, 3.0
    r1 = one_gate_dm(orc, X, "DECOHERENCE", 0.0, t1=t1, t2=t2, tgate=tg)
    assert abs(r1[1, 1] - math.exp(-tg / t1)) < 1e-15
    rp = one_gate_dm(orc, H, "DECOHERENCE", 0.0, t1=t1, t2=t2, tgate=tg)
    assert abs(abs(rp[0, 1]) - 0.5 * math.exp(-tg / t2)) < 1e-15


def test_trajectory_choice_rule(orc):
    """Damping on |1>: the trajectory decays to |0> exactly when the draw is at
    least the no-decay weight 1 - p; rotation error adds e (2u - 1) to theta."""
    p = 0.3
    rules = w.noise_rules([w.noise_rule("DAMPING", "X", p)])
    for seed in range(30):
        st, nd = orc.run_noisy(1, w.pack([G("X", 0)]), rules, seed=seed)
        u = u01(orc, seed, 0)
        want = np.array([1, 0]) if u >= 1 - p else np.array([0, 1])
        assert nd == 1 and np.max(np.abs(orc.as_complex(st) - want)) < 1e-15
    th, e = 0.7, 0.05
    for seed in range(5):
        st, nd = orc.run_noisy(1, w.pack([G("RX", 0, theta=th)]), w.noise_rules([]), rot_err=e, seed=seed)
        d = e * (2 * u01(orc, seed, 0) - 1)
        ref = orc.run(1, w.pack([G("RX", 0, theta=th + d)]))
        assert nd == 1 and np.array_equal(st, ref)


def test_noiseless_rules_leave_the_circuit(orc):
    n = 4
    g = w.random_circuit(n, 60, 3)
    rules = w.noise_rules([w.noise_rule("DEPOLARIZING", None, 0.0), w.noise_rule("DAMPING", "CNOT", 0.0)])
    st, nd = orc.run_noisy(n, g, rules, seed=1)
    assert np.max(np.abs(st - orc.run(n, g))) < 1e-14
    touched = sum(2 if r["type"] in (12, 13, 14) else 1 for r in g)
    assert nd == touched + sum(2 for r in g if r["type"] == 12)


def test_trajectory_average_is_the_density_matrix(orc):
    n = 3
    g = w.pack([G("H", 0), G("CNOT", 0, 1), G("RX", 2, theta=1.1), G("CZ", 1, 2), G("T", 0), G("H", 2)])
    rules = w.noise_rules([w.noise_rule("DAMPING", "CNOT", 0.2), w.noise_rule("DEPOLARIZING", None, 0.1),
                           w.noise_rule("DECOHERENCE", "H", t1=30.0, t2=20.0, tgate=4.0),
                           w.noise_rule("BITPHASEFLIP", "CZ", 0.15, q0=1, q1=2)])
    rho = orc.dm_run(n, g, rules)
    K = 4000
    acc = np.zeros((8, 8), dtype=np.complex128)
    for seed in range(K):
        st, _ = orc.run_noisy(n, g, rules, seed=seed)
        v = orc.as_complex(st)
        acc += np.outer(v, v.conj())
    acc /= K
    assert abs(np.trace(rho) - 1) < 1e-14
    assert np.max(np.abs(acc - rho)) < 5 * 0.5 / math.sqrt(K)


def test_readout_error(orc):
    n, shots, f0, f1, seed = 5, 20000, 0.9, 0.85, 4
    zeros = orc.readout(np.zeros(shots, dtype=np.uint64), n, f0, f1, seed)
    ones = orc.readout(np.full(shots, (1 << n) - 1, dtype=np.uint64), n, f0, f1, seed)
    for s in range(20):
        for i in range(n):
            u = u01(orc, seed, s * n + i)
            assert ((int(zeros[s]) >> i) & 1) == (1 if u >= f0 else 0)
            assert ((int(ones[s]) >> i) & 1) == (0 if u >= f1 else 1)
    flips0 = sum(bin(int(x)).count("1") for x in zeros) / (shots * n)
    flips1 = 1 - sum(bin(int(x)).count("1") for x in ones) / (shots * n)
    for f, q in ((flips0, 1 - f0), (flips1, 1 - f1)):
        assert abs(f - q) < 5 * math.sqrt(q * (1 - q) / (shots * n))
