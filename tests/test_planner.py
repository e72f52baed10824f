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


def check_plan(q, orc, n, gates, params=None, make=None):
    p = q.qs_plan_create(n, gates, q.PLAN_GREEDY, 5) if make is None else make(n, gates)
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


def apply_pass_ops(orc, st, n, qmask, ops, tables):
    """Applies a pass's op list (qs_plan_pass_ops) to a state on the host: 2x2 ops
    through the oracle, phase tables by their definition."""
    st = orc.as_complex(st).copy()
    qs_ = [b for b in range(n) if (qmask >> b) & 1]
    x = np.arange(1 << n)
    j = np.zeros(1 << n, dtype=np.int64)
    for pos, b in enumerate(qs_):
        j |= ((x >> b) & 1) << pos
    for o in ops:
        if o["kind"] == 0:
            st = orc.as_complex(orc.apply_matrix(st, n, [o["target"]], o["m"], o["ctrl_mask"]))
        else:
            assert o["bits"] == len(qs_)
            st = st * tables[o["table"]][j]
            for qo, qt in o.get("signs", []):   # (-1)^(x_qo x_qt): a CZ the table absorbed
                assert not (qmask >> qo) & 1 and (qmask >> qt) & 1
                st = st * np.where((x >> qo) & (x >> qt) & 1, -1.0, 1.0)
    return st


def chain_circuit(n, seed):
    rng = w.SplitMix64(seed)
    recs = []
    for _ in range(50):
        t = rng.below(n)
        c = (t + 1 + rng.below(n - 1)) % n
        k = rng.below(6)
        if k < 3:
            for _ in range(2 + rng.below(3)):
                name = w.ONE_QUBIT[rng.below(len(w.ONE_QUBIT))]
                recs.append(w.gate(name, t, theta=rng.angle(), phi=rng.angle(), lam=rng.angle(),
                                   ctrl_mask=(1 << c) if k == 2 else 0))
        elif k == 3:
            recs.append(w.gate("RZ", t, theta=rng.angle()))
            recs.append(w.gate("CZ", c, t) if rng.below(2) else w.gate("CNOT", t, c))
            recs.append(w.gate("T", t))
        else:
            recs.append(w.gate(("CNOT", "CZ", "CR")[rng.below(3)], c, t, theta=rng.angle()))
    return w.pack(recs)


@pytest.mark.parametrize("tables", [True, False])
@pytest.mark.parametrize("aggregate", [True, False])
def test_pass_op_lists_compose_to_their_passes(q, orc, tables, aggregate):
    """Every tile pass's op list (after aggregation and the split of general ops
    into real rotations and phase tables) applied to a random state equals the
    pass's gates applied in order (oracle), 1e-13."""
    cases = [(10, w.layered_u3_cz(10, 8, 2), None), (9, w.random_circuit(9, 300, 4), None),
             (15, w.layered_u3_cz(15, 10, 2), None), (15, w.random_circuit(15, 300, 7, two_qubit_prob=0.4), None),
             (8, chain_circuit(8, 5), None), (7, w.hea_ansatz(7, 3)[0], w.uniform_angles(200, 6)),
             (5, w.random_circuit(5, 200, 8, two_qubit_prob=0.4), None), (3, chain_circuit(3, 9), None)]
    q.qs_set_phase_tables(tables)
    q.qs_set_aggregate(aggregate)
    try:
        for (n, g, params), lookahead in [(c, la) for c in cases for la in (False, True)]:
            p = q.qs_plan_create_variant(n, g, max(4, min(n, 12)), 2) if lookahead else \
                q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
            try:
                st = w.random_state(n, 17 + n)
                st = st / np.sqrt(np.sum(st * st))
                for i, (kind, qm, idx) in enumerate(q.qs_plan_passes(p)):
                    ops, tabs = q.qs_plan_pass_ops(p, i, g, params)
                    want = orc.as_complex(orc.apply_circuit(st.copy(), n, g[idx], params))
                    got = apply_pass_ops(orc, st, n, qm if kind == 1 else 0, ops, tabs)
                    assert np.max(np.abs(got - want)) < 1e-13, (n, i)
                    st = want.view(np.float64).copy()
            finally:
                q.qs_plan_free(p)
    finally:
        q.qs_set_phase_tables(True)
        q.qs_set_aggregate(True)


def _general(m):
    return np.all(np.abs(m) > 0) and np.any(np.abs(m.imag) > 0)


def test_phase_tables_turn_brickwork_layers_real(q):
    """On the brickwork every uncontrolled general op of a tile pass becomes a
    real rotation, with about one phase table per layer."""
    n = 12
    g = w.layered_u3_cz(n, 10, 3)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    try:
        tables = general = real = 0
        for i, (kind, qm, idx) in enumerate(q.qs_plan_passes(p)):
            ops, tabs = q.qs_plan_pass_ops(p, i, g)
            tables += sum(1 for o in ops if o["kind"] == 1)
            for o in ops:
                if o["kind"] == 0 and o["ctrl_mask"] == 0:
                    general += _general(o["m"])
                    real += bool(np.all(np.abs(o["m"].imag) == 0) and np.all(np.abs(o["m"]) > 0))
        assert general == 0 and real >= 10 * n * 0.9 and 5 <= tables <= 15
    finally:
        q.qs_plan_free(p)


def u3_params(M):
    """(theta, phi, lambda) of the U3 equal to the 2x2 unitary M up to a global phase."""
    th = 2 * np.arctan2(abs(M[1, 0]), abs(M[0, 0]))
    g0 = np.angle(M[0, 0]) if abs(M[0, 0]) > 1e-12 else np.angle(-M[0, 1]) if abs(M[0, 1]) > 0 else 0.0
    phi = np.angle(M[1, 0]) - g0 if abs(M[1, 0]) > 1e-12 else 0.0
    lam = np.angle(-M[0, 1]) - g0 if abs(M[0, 1]) > 1e-12 else np.angle(M[1, 1]) - g0 - phi
    return th, phi, lam


def test_nearly_antidiagonal_products_split_exactly(q, orc):
    """Pairs of U3 gates whose product is X (or Y) up to a phase: the aggregated op
    has diagonal entries that are rounding noise, independent in a and d.  Its
    split into phases and a real rotation must still reproduce it (1e-13)."""
    n = 5
    rng = np.random.Generator(np.random.PCG64(3))
    recs = []
    for rep in range(3):
        for k in range(n):
            th, ph, la = rng.uniform(0.1, 3.0, 3)
            V = orc.gate_matrix(w.pack([w.gate("U3", 0, theta=th, phi=ph, lam=la)])[0], 1)[2]
            T = np.array([[0, 1], [1, 0]]) if (k + rep) % 2 else np.array([[0, -1j], [1j, 0]])
            W = T @ V.conj().T
            recs.append(w.gate("U3", k, theta=th, phi=ph, lam=la))
            recs.append(w.gate("U3", k, *[], **dict(zip(("theta", "phi", "lam"), u3_params(W)))))
        recs += [w.gate("CZ", k, k + 1) for k in range(rep % 2, n - 1, 2)]
    g = w.pack(recs)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    try:
        st = w.random_state(n, 4)
        st = st / np.sqrt(np.sum(st * st))
        for i, (kind, qm, idx) in enumerate(q.qs_plan_passes(p)):
            ops, tabs = q.qs_plan_pass_ops(p, i, g)
            want = orc.as_complex(orc.apply_circuit(st.copy(), n, g[idx]))
            got = apply_pass_ops(orc, st, n, qm if kind == 1 else 0, ops, tabs)
            assert np.max(np.abs(got - want)) < 1e-13, i
            st = want.view(np.float64).copy()
    finally:
        q.qs_plan_free(p)


def test_tables_absorb_cz_across_tile_boundaries(q):
    """On the n=30 brickwork every CZ with one qubit outside its pass's tile is a
    sign term of a phase table, and the in-tile CZs ahead of each qubit's next
    rotation join the tables too: few controlled diagonal ops remain."""
    n = 30
    g = w.layered_u3_cz(n, 20, 1)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    try:
        signs = left = 0
        for i, (kind, qm, idx) in enumerate(q.qs_plan_passes(p)):
            ops, _ = q.qs_plan_pass_ops(p, i, g)
            for o in ops:
                if o["kind"] == 1:
                    signs += len(o["signs"])
                elif o["ctrl_mask"] and abs(o["m"][0, 1]) == 0:
                    left += 1
        assert signs >= 140 and left <= 30, (signs, left)
    finally:
        q.qs_plan_free(p)


def shipped_scorer(orc):
    """The shipped cost model's forward pass on the host (the oracle's perceptron)."""
    import json
    import os
    import paper_2212_14201_gb300 as pkg
    path = os.path.join(os.path.dirname(pkg.__file__), "costmodel_weights.json")
    with open(path) as f:
        d = json.load(f)
    wts = np.asarray(d["weights"], dtype=np.float64)
    return lambda x: orc.mlp_forward(d["features"], d["hidden"], wts, x)


@pytest.mark.parametrize("n,maker,seed", [(13, "random", 2), (16, "random", 3), (14, "layered", 4), (16, "layered", 5)])
def test_lookahead_plans_are_valid_reorderings(q, orc, n, maker, seed):
    """Strategy 2 (the greedy pass or a variant kept off one of its qubits) keeps
    every gate exactly once in a commuting order: the replay equals the program."""
    g = w.random_circuit(n, 500, seed, two_qubit_prob=0.4) if maker == "random" else w.layered_u3_cz(n, 16, seed)
    for m in (8, 11):
        check_plan(q, orc, n, g, make=lambda nn, gg: q.qs_plan_create_variant(nn, gg, m, 2))


def test_lookahead_absorbs_more_per_pass(q):
    """On brickwork (config 1's structure: n=30, 20 layers of U3 + CZ) and on the
    n=32 random workload, the lookahead passes cover the program in fewer passes
    than the program-order greedy passes (20 -> 13 and 36 -> 32 at width 12)."""
    for n, g in ((30, w.layered_u3_cz(30, 20, 1)), (32, w.random_circuit(32, 2000, 2, two_qubit_prob=0.4))):
        counts = []
        for strategy in (0, 2):
            p = q.qs_plan_create_variant(n, g, 12, strategy)
            try:
                counts.append(q.qs_plan_get_stats(p)["n_passes"])
            finally:
                q.qs_plan_free(p)
        assert counts[1] < counts[0], (n, counts)


@pytest.mark.parametrize("n,maker,seed", [(14, "random", 6), (16, "layered", 7)])
def test_scored_plans_are_valid_reorderings(q, orc, n, maker, seed):
    """The learned planner driven by a host cost model (qs_plan_create_scored):
    whatever it chooses is a valid reordering, with tile passes of at most 12
    qubits holding the low qubits."""
    g = w.random_circuit(n, 500, seed, two_qubit_prob=0.4) if maker == "random" else w.layered_u3_cz(n, 16, seed)
    sc = shipped_scorer(orc)
    check_plan(q, orc, n, g, make=lambda nn, gg: q.qs_plan_create_scored(nn, gg, sc))
    # a cost model that charges every pass alike prefers the candidates that absorb the most
    flat = lambda x: np.zeros(len(x))
    check_plan(q, orc, n, g, make=lambda nn, gg: q.qs_plan_create_scored(nn, gg, flat))


def test_scored_planner_judge_and_choices(q, orc):
    """The planner around a cost model (planning only, host forward passes):
    - with the shipped model, on the n=32 random workload (2000 gates, seed 2), an
      n=28 brickwork and config 1's brickwork (n=30, 20 layers), every learned plan
      holds every gate exactly once and is never predicted slower than the greedy
      plan (the judge keeps the greedy passes unless the model's own are predicted
      5 % faster);
    - with a model that charges every pass alike, the planner prefers the
      candidates that absorb the most gates over two passes: on the n=32 workload it
      plans at least 5 % fewer passes than greedy and keeps them (no fallback)."""
    sc = shipped_scorer(orc)
    flat = lambda x: np.zeros(len(x))

    def predicted(score, p, g):
        return float(np.sum(np.exp(score(q.qs_plan_features(p, g)))))

    cases = ((32, w.random_circuit(32, 2000, 2, two_qubit_prob=0.4)), (28, w.layered_u3_cz(28, 12, 301)),
             (30, w.layered_u3_cz(30, 20, 1)))
    for n, g in cases:
        pl = q.qs_plan_create_scored(n, g, sc)
        pg = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
        try:
            order = np.concatenate([idx for _, _, idx in q.qs_plan_passes(pl)])
            assert sorted(order.tolist()) == list(range(len(g)))
            assert predicted(sc, pl, g) <= predicted(sc, pg, g) * (1 + 1e-12)
        finally:
            q.qs_plan_free(pl)
            q.qs_plan_free(pg)
    n, g = cases[0]
    pl = q.qs_plan_create_scored(n, g, flat)
    pg = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    try:
        sl, sg = q.qs_plan_get_stats(pl), q.qs_plan_get_stats(pg)
        assert sl["learned_fallback"] == 0 and sl["n_passes"] <= 0.95 * sg["n_passes"], (sl, sg)
    finally:
        q.qs_plan_free(pl)
        q.qs_plan_free(pg)


def test_scorer_failure_is_reported(q):
    def bad(x):
        raise RuntimeError("no model")
    with pytest.raises(q.QsimError):
        q.qs_plan_create_scored(8, w.random_circuit(8, 50, 1), bad)


@pytest.mark.parametrize("n,maker,seed", [(30, "layered", 1), (16, "layered", 2), (20, "random", 3), (12, "chain", 4)])
def test_kernel_ops_cover_the_pass_ops(q, n, maker, seed):
    """The tile engine's op slots for each pass (qs_plan_pass_kernel_ops) account for
    the pass's op list (qs_plan_pass_ops) exactly: every phase table once (as its
    own sweep, inside a rotation group's loop, or in the tile's load or store loop),
    every in-tile uncontrolled real rotation in exactly one group of four, three or
    two or as a single rotation, and 12 limb products per amplitude for each group,
    single rotation and table."""
    g = {"layered": lambda: w.layered_u3_cz(n, 20, seed),
         "random": lambda: w.random_circuit(n, 400, seed, two_qubit_prob=0.4),
         "chain": lambda: chain_circuit(n, seed)}[maker]()
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    try:
        for i, (kind, qm, idx) in enumerate(q.qs_plan_passes(p)):
            c, ipa = q.qs_plan_pass_kernel_ops(p, i, g)
            if kind != 1:
                assert not c.any() and ipa == 0.0
                continue
            ops, _ = q.qs_plan_pass_ops(p, i, g)
            tables = sum(1 for o in ops if o["kind"] == 1)
            reals = sum(1 for o in ops if o["kind"] == 0 and o["ctrl_mask"] == 0 and (qm >> o["target"]) & 1
                        and np.all(np.imag(o["m"]) == 0) and o["m"][0, 0] != 0 and o["m"][0, 1] != 0)
            assert c[10] == tables, (i, c, tables)
            assert 4 * c[14] + 3 * c[13] + 2 * c[11] + c[4] == reals, (i, c, reals)
            assert 0 <= c[0] <= c[10]
            # tables in rotation-group loops: at most one per group; in load/store: at most two
            assert c[0] <= c[11] + c[13] + c[14] + 2
            grouped = c[14] + c[13] + c[11] + c[4] + c[10]
            assert ipa >= 12.0 * grouped - 1e-9
    finally:
        q.qs_plan_free(p)


def test_features_of_parametrised_programs(q):
    """Pass features need no parameters: a parametrised program (every rotation
    reads a parameter) is featurised with generic angles, and gives the features of
    the same program with generic explicit angles in its records; the kernel-op
    part of every tile pass is filled in (at least one shared-memory sweep; limb
    products where it has rotations)."""
    n = 14
    g, npar = w.hea_ansatz(n, 3)
    explicit = g.copy()
    for r in explicit:
        if r["param_idx"] >= 0:
            r["p"][0], r["p"][1], r["p"][2] = 1.1, 0.4, 2.3
            r["param_idx"] = -1
    p1 = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    p2 = q.qs_plan_create(n, explicit, q.PLAN_GREEDY, 5)
    try:
        f1, f2 = q.qs_plan_features(p1, g), q.qs_plan_features(p2, explicit)
        assert f1.shape == (q.qs_plan_get_stats(p1)["n_passes"], q._lib.PASS_FEATURES) and f1.shape == f2.shape
        assert np.array_equal(f1, f2)
        tile = f1[f1[:, 0] == 1.0]
        assert len(tile) >= 1 and np.any(tile[:, 14] > 0) and np.all(tile[:, 24] > 0)
        gate = f1[f1[:, 0] == 0.0]
        assert np.all(gate[:, 14:] == 0.0)
    finally:
        q.qs_plan_free(p1)
        q.qs_plan_free(p2)
