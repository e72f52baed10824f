"""Host-side checks of the greedy fusion planner (no GPU): every plan is a valid
reordering of the program -- replaying its execution order on the CPU oracle
gives the program's state -- and each tile pass respects the tile rules."""
import numpy as np
import pytest

import workloads as w


@pytest.fixture(scope="module")
def q():
    import paper_2212_14201_gb300 as q
    q.build()
    return q


DIAG = {w.GATE_CODES[k] for k in ("I", "Z", "S", "T", "RZ", "P", "CZ", "CR")}
TWO = {w.GATE_CODES[k] for k in ("CNOT", "CZ", "CR")}


def target_of(rec):
    return int(rec["q1"]) if int(rec["type"]) in TWO else int(rec["q0"])


def check_plan(q, orc, n, gates, params=None):
    p = q.qs_plan_create(n, gates, q.PLAN_GREEDY, 5)
    try:
        passes = q.qs_plan_passes(p)
        stats = q.qs_plan_get_stats(p)
    finally:
        q.qs_plan_free(p)
    order = np.concatenate([g for _, _, g in passes])
    assert sorted(order.tolist()) == list(range(len(gates)))   # every gate exactly once
    for kind, qm, idx in passes:
        if kind == 1:
            assert bin(qm).count("1") <= min(n, 12)
            assert qm & ((1 << min(n, 3)) - 1) == (1 << min(n, 3)) - 1
            for k in idx:
                if int(gates[k]["type"]) not in DIAG:
                    assert (qm >> target_of(gates[k])) & 1
        else:
            assert len(idx) == 1
    ref = orc.run(n, gates, params)
    re = orc.run(n, gates[order], params)
    assert np.max(np.abs(ref - re)) < 1e-12
    return stats


@pytest.mark.parametrize("n,ng,seed,p2", [(3, 60, 0, None), (8, 300, 1, None), (13, 400, 2, 0.4), (16, 500, 3, 0.4),
                                          (14, 600, 4, 0.8)])
def test_random_plans_are_valid_reorderings(q, orc, n, ng, seed, p2):
    check_plan(q, orc, n, w.random_circuit(n, ng, seed, two_qubit_prob=p2))


def test_brickwork_plan_fuses(q, orc):
    n = 16
    g = w.layered_u3_cz(n, 20, 1)
    st = check_plan(q, orc, n, g)
    assert st["n_tile_passes"] >= 1 and st["n_passes"] < len(g) / 5


def test_controls_and_diagonals_outside_tiles(q, orc):
    n = 15
    recs = []
    rng = w.SplitMix64(3)
    for i in range(300):
        t = rng.below(n)
        c1 = (t + 1 + rng.below(n - 1)) % n
        c2 = (c1 + 1 + rng.below(n - 2)) % n
        if c2 == t:
            c2 = (c2 + 1) % n
        kind = i % 5
        if kind == 0:
            recs.append(w.gate("X", t, ctrl_mask=(1 << c1) | (1 << c2)))   # Toffoli
        elif kind == 1:
            recs.append(w.gate("CR", c1, t, theta=rng.angle()))
        elif kind == 2:
            recs.append(w.gate("U3", t, theta=rng.angle(), phi=rng.angle(), lam=rng.angle(), ctrl_mask=1 << c1))
        elif kind == 3:
            recs.append(w.gate("RZ", t, theta=rng.angle(), ctrl_mask=1 << c2))
        else:
            recs.append(w.gate("H", t))
    check_plan(q, orc, n, w.pack(recs))


def test_plan_rejects_other_program(q):
    g = w.random_circuit(6, 40, 1)
    p = q.qs_plan_create(6, g, q.PLAN_GREEDY, 5)
    try:
        with pytest.raises(q.QsimError):
            q.qs_apply(0, w.random_circuit(6, 40, 2), None, p)   # NULL state is rejected first
    finally:
        q.qs_plan_free(p)
