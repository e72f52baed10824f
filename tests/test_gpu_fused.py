"""GPU parity of the fused path (greedy plan: shared-memory tile passes) against
the CPU oracle, and fused-vs-plain agreement at the full n=30 benchmark size."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available()
    import paper_2212_14201_gb300 as q
    q.build()
    return q


@pytest.fixture(params=["fp64", "q60"])
def arith(request, q):
    return {"fp64": q.ARITH_FP64, "q60": q.ARITH_FIXED}[request.param]


def fused(q, n, gates, params=None, init=None, arith=None):
    p = q.qs_plan_create(n, gates, q.PLAN_GREEDY, 5)
    h = q.qs_alloc(n)
    try:
        if arith is not None:
            q.qs_set_arith(h, arith)
        if init is not None:
            q.qs_set_state(h, np.ascontiguousarray(init, dtype=np.complex128))
        q.qs_apply(h, gates, params, p)
        return q.qs_get_state(h), q.qs_plan_get_stats(p)
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)


@pytest.mark.parametrize("n,ng,seed,p2", [(1, 30, 0, None), (3, 80, 1, None), (7, 200, 2, None), (12, 200, 0, None),
                                          (13, 400, 3, 0.4), (15, 500, 4, 0.4), (19, 600, 5, 0.4), (22, 400, 6, 0.4)])
def test_fused_random_circuits(q, orc, arith, n, ng, seed, p2):
    g = w.random_circuit(n, ng, seed, two_qubit_prob=p2)
    psi, st = fused(q, n, g, arith=arith)
    assert np.max(np.abs(psi - orc.as_complex(orc.run(n, g)))) < TOL


def _table_edge_programs(n, seed):
    """(a) diagonal gates only: one tile pass whose only kernel op is a phase table;
    (b) RZ, RY and RZ layers (and CZs): a pass opened and closed by a table."""
    rng = w.SplitMix64(seed)
    a = [w.gate("RZ", k, theta=rng.angle()) for k in range(n)] + [w.gate("CZ", k, k + 1) for k in range(0, n - 1, 2)] + \
        [w.gate("T", k) for k in range(0, n, 3)]
    b = [w.gate("RZ", k, theta=rng.angle()) for k in range(n)] + [w.gate("RY", k, theta=rng.angle()) for k in range(n)] + \
        [w.gate("RZ", k, theta=rng.angle()) for k in range(n)] + [w.gate("CZ", k, k + 1) for k in range(1, n - 1, 2)]
    return w.pack(a), w.pack(b)


@pytest.mark.parametrize("n", [6, 14, 20])
def test_phase_tables_in_load_and_store_loops(q, orc, n):
    """Q60 passes whose phase tables run in the tile's load and store loops: a pass
    whose only op is such a table (no shared-memory op at all), a pass opened and
    closed by one, and the two programs applied one after the other to the same
    state, against the oracle within 1e-12."""
    ga, gb = _table_edge_programs(n, n)
    pa = q.qs_plan_create(n, ga, q.PLAN_GREEDY, 5)
    pb = q.qs_plan_create(n, gb, q.PLAN_GREEDY, 5)
    h = q.qs_alloc(n)
    try:
        c, _ = q.qs_plan_pass_kernel_ops(pa, 0, ga)
        assert c[0] >= 1                      # the table rides in a load or store loop
        if n == 6:
            assert c[1:].sum() - c[0] == 0    # and the pass has no other op
        c, _ = q.qs_plan_pass_kernel_ops(pb, 0, gb)
        assert c[0] >= 2
        q.qs_set_arith(h, q.ARITH_FIXED)
        q.qs_apply(h, ga, None, pa)
        assert np.max(np.abs(q.qs_get_state(h) - orc.as_complex(orc.run(n, ga)))) < TOL
        q.qs_set_zero(h)
        q.qs_apply(h, gb, None, pb)
        assert np.max(np.abs(q.qs_get_state(h) - orc.as_complex(orc.run(n, gb)))) < TOL
        init = w.random_state_fast(n, 5)
        init = init / np.sqrt(np.sum(init * init))
        q.qs_set_state(h, orc.as_complex(init))
        q.qs_apply(h, ga, None, pa)
        q.qs_apply(h, gb, None, pb)
        want = orc.as_complex(orc.apply_circuit(orc.apply_circuit(init.copy(), n, ga), n, gb))
        assert np.max(np.abs(q.qs_get_state(h) - want)) < TOL
    finally:
        q.qs_free(h)
        q.qs_plan_free(pa)
        q.qs_plan_free(pb)


@pytest.mark.parametrize("n", [12, 14, 17, 21])
def test_fused_brickwork(q, orc, arith, n):
    g = w.layered_u3_cz(n, 20, 1)
    psi, st = fused(q, n, g, arith=arith)
    assert st["n_tile_passes"] >= 1
    assert np.max(np.abs(psi - orc.as_complex(orc.run(n, g)))) < TOL


def test_fused_controls_outside_tiles(q, orc, arith):
    n = 18
    rng = w.SplitMix64(7)
    recs = []
    for i in range(400):
        t = rng.below(n)
        c = (t + 1 + rng.below(n - 1)) % n
        d = (c + 1 + rng.below(n - 2)) % n
        if d == t:
            d = (d + 1) % n
        k = i % 6
        if k == 0:
            recs.append(w.gate("X", t, ctrl_mask=(1 << c) | (1 << d)))
        elif k == 1:
            recs.append(w.gate("CR", c, t, theta=rng.angle()))
        elif k == 2:
            recs.append(w.gate("U3", t, theta=rng.angle(), phi=rng.angle(), lam=rng.angle(), ctrl_mask=1 << c))
        elif k == 3:
            recs.append(w.gate("T", t, ctrl_mask=1 << d, dagger=1))
        elif k == 4:
            recs.append(w.gate("Y", t, ctrl_mask=1 << c))
        else:
            recs.append(w.gate("RX", t, theta=rng.angle()))
    g = w.pack(recs)
    init = w.random_state_fast(n, 3)
    init /= np.linalg.norm(init)
    psi, _ = fused(q, n, g, init=init.view(np.complex128), arith=arith)
    ref = orc.as_complex(orc.apply_circuit(init.copy(), n, g))
    assert np.max(np.abs(psi - ref)) < TOL


def test_fused_parametrised_plan_reused_across_params(q, orc):
    n = 14
    g, npar = w.hea_ansatz(n, 4)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    h = q.qs_alloc(n)
    try:
        for seed in (1, 2):
            th = w.uniform_angles(npar, seed)
            q.qs_set_zero(h)
            q.qs_apply(h, g, th, p)
            assert np.max(np.abs(q.qs_get_state(h) - orc.as_complex(orc.run(n, g, th)))) < TOL
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)


def test_full_size_fused_vs_plain_and_invariants(q):
    """n=30, depth-20 brickwork (the benchmark workload, its launch configuration):
    fused and plain agree amplitude by amplitude on a sample; the norm stays 1;
    after one layer <Z_i> = cos(theta_i) (CZ commutes with Z)."""
    import torch
    n = 30
    g = w.layered_u3_cz(n, 20, 1)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    a = q.qs_alloc(n)
    try:
        q.qs_apply(a, g[:45], None, None)
        ez = q.qs_expect_z_all(a)
        assert np.max(np.abs(ez - np.cos(g["p"][:n, 0]))) < TOL
        q.qs_set_zero(a)
        q.qs_apply(a, g, None, p)
        assert abs(q.qs_probs(a, [])[0] - 1.0) < TOL
        idx = torch.randint(0, 1 << n, (1 << 16,), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
        amps = torch.empty(2 << n, dtype=torch.float64, device="cuda")
        q.qs_get_state(a, amps)
        fz = amps.view(torch.complex128)[idx].clone()
        del amps
        torch.cuda.empty_cache()
        q.qs_set_zero(a)
        q.qs_apply(a, g, None, None)
        amps = torch.empty(2 << n, dtype=torch.float64, device="cuda")
        q.qs_get_state(a, amps)
        pl = amps.view(torch.complex128)[idx]
        assert float((fz - pl).abs().max()) < TOL
        del amps
    finally:
        q.qs_free(a)
        q.qs_plan_free(p)


def _amp_errors(got, ref, chunk=1 << 24):
    """max |got - ref|, and max |got - ref| / |ref| over entries with |ref| >= 2^-20,
    in chunks (the full n=30 arrays are 16 GiB each)."""
    mabs = 0.0
    mrel = 0.0
    for o in range(0, got.size, chunk):
        a = got[o:o + chunk]
        b = ref[o:o + chunk]
        d = np.abs(a - b)
        mabs = max(mabs, float(d.max()))
        ab = np.abs(b)
        big = ab >= 2.0 ** -20
        if np.any(big):
            mrel = max(mrel, float((d[big] / ab[big]).max()))
    return mabs, mrel


def test_config1_full_state_against_oracle_n30(q, orc):
    """The benchmark workload at its full size (n=30, depth-20 U3 + CZ brickwork,
    890 gates, seed 1): every one of the 2^30 amplitudes of the fused Q60 path
    (greedy plan, the benchmark's launch configuration), of plain per-gate Q60
    and of plain per-gate FP64 within 1e-12 of the CPU oracle's state."""
    n = 30
    g = w.layered_u3_cz(n, 20, 1)
    ref = orc.as_complex(orc.run(n, g))
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    h = q.qs_alloc(n)
    got = np.empty(1 << n, dtype=np.complex128)
    try:
        results = {}
        for name, plan, arith in (("fused_q60", p, q.ARITH_FIXED), ("plain_q60", None, q.ARITH_FIXED),
                                  ("plain_fp64", None, q.ARITH_FP64)):
            q.qs_set_zero(h)
            q.qs_set_arith(h, arith)
            q.qs_apply(h, g, None, plan)
            q.qs_get_state(h, got)
            results[name] = _amp_errors(got, ref)
            print(f"n=30 config-1 {name}: max abs err {results[name][0]:.3e}, "
                  f"max rel err (|a|>=2^-20) {results[name][1]:.3e}")
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)
    for name, (mabs, _) in results.items():
        assert mabs < TOL, name


def test_q60_tile_engine_all_widths(q, orc):
    """The Q60 tile engine against the oracle on random circuits with controls
    inside and outside the tiles, the brickwork, the ansatz, and every tile width
    4..13."""
    cases = [(13, w.random_circuit(13, 400, 3, two_qubit_prob=0.4), None),
             (17, w.layered_u3_cz(17, 12, 1), None), (16, w.random_circuit(16, 300, 8), None),
             (15, w.hea_ansatz(15, 4)[0], w.uniform_angles(120, 3)), (9, run_chain_circuit(9, 4), None)]
    for n, g, th in cases:
        p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
        h = q.qs_alloc(n)
        try:
            q.qs_set_arith(h, q.ARITH_FIXED)
            q.qs_apply(h, g, th, p)
            psi = q.qs_get_state(h)
        finally:
            q.qs_free(h)
            q.qs_plan_free(p)
        assert np.max(np.abs(psi - orc.as_complex(orc.run(n, g, th)))) < TOL, n
    for m in range(4, 14):
        n = 15
        g = w.random_circuit(n, 300, 30 + m, two_qubit_prob=0.4)
        p = q.qs_plan_create_tiled(n, g, m)
        h = q.qs_alloc(n)
        try:
            q.qs_set_arith(h, q.ARITH_FIXED)
            q.qs_apply(h, g, None, p)
            psi = q.qs_get_state(h)
        finally:
            q.qs_free(h)
            q.qs_plan_free(p)
        assert np.max(np.abs(psi - orc.as_complex(orc.run(n, g)))) < TOL, m


def run_chain_circuit(n, seed):
    """Runs of one-qubit gates on one qubit (some with the same extra control),
    self-cancelling pairs (H H, X X, S then S-dagger), diagonal gates separated by
    gates they commute with (CZ, a CNOT controlled on the same qubit) and a
    two-qubit gate now and then: material for the aggregation of a pass's gates
    into fewer unitaries."""
    rng = w.SplitMix64(seed)
    recs = []
    for _ in range(60):
        t = rng.below(n)
        c = (t + 1 + rng.below(n - 1)) % n
        k = rng.below(8)
        if k < 4:
            cm = (1 << c) if k == 3 else 0
            for _ in range(2 + rng.below(4)):
                name = w.ONE_QUBIT[rng.below(len(w.ONE_QUBIT))]
                recs.append(w.gate(name, t, theta=rng.angle(), phi=rng.angle(), lam=rng.angle(), ctrl_mask=cm))
        elif k == 4:
            name = ("H", "X", "S")[rng.below(3)]
            recs.append(w.gate(name, t))
            recs.append(w.gate(name, t, dagger=1))
        elif k == 5:
            recs.append(w.gate("RZ", t, theta=rng.angle()))
            recs.append(w.gate("CZ", c, t) if rng.below(2) else w.gate("CNOT", t, c))
            recs.append(w.gate("T", t))
            recs.append(w.gate("P", t, theta=rng.angle()))
        else:
            recs.append(w.gate(("CNOT", "CZ", "CR")[rng.below(3)], c, t, theta=rng.angle()))
    return w.pack(recs)


@pytest.mark.parametrize("n", [3, 9, 14])
def test_aggregation_matches_oracle_and_reduces_work(q, orc, arith, n):
    """Fused apply with gate aggregation on and off against the oracle (1e-12),
    and the aggregated passes do fewer limb products / flops (timing log)."""
    g = run_chain_circuit(n, 40 + n)
    ref = orc.as_complex(orc.run(n, g))
    work = {}
    try:
        for on in (True, False):
            q.qs_set_aggregate(on)
            p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
            h = q.qs_alloc(n)
            try:
                q.qs_set_arith(h, arith)
                q.qs_timing_enable(h, True)
                q.qs_apply(h, g, None, p)
                recs = q.qs_timing_fetch(h)
                got = q.qs_get_state(h)
            finally:
                q.qs_free(h)
                q.qs_plan_free(p)
            assert np.max(np.abs(got - ref)) < TOL, on
            work[on] = sum(r["int_ops"] + r["flops"] for r in recs if r["kind"] == q._lib.K_TILE)
    finally:
        q.qs_set_aggregate(True)
    assert work[True] < 0.9 * work[False]


@pytest.mark.parametrize("n,kind", [(13, "brick"), (14, "rand"), (12, "hea"), (9, "chain")])
def test_phase_tables_match_oracle_and_cut_work(q, orc, n, kind):
    """Q60 tile passes with the general ops split into real rotations and phase
    tables, against the oracle (1e-12) and against the switch off; on the
    brickwork the limb products per step drop."""
    g = {"brick": lambda: w.layered_u3_cz(n, 12, 4), "rand": lambda: w.random_circuit(n, 400, 11),
         "hea": lambda: w.hea_ansatz(n, 4)[0], "chain": lambda: run_chain_circuit(n, 77)}[kind]()
    params = w.uniform_angles(400, 3)
    ref = orc.as_complex(orc.run(n, g, params))
    work = {}
    try:
        for on in (True, False):
            q.qs_set_phase_tables(on)
            p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
            h = q.qs_alloc(n)
            try:
                q.qs_set_arith(h, q.ARITH_FIXED)
                q.qs_timing_enable(h, True)
                q.qs_apply(h, g, params, p)
                recs = q.qs_timing_fetch(h)
                got = q.qs_get_state(h)
            finally:
                q.qs_free(h)
                q.qs_plan_free(p)
            assert np.max(np.abs(got - ref)) < TOL, on
            work[on] = sum(r["int_ops"] for r in recs if r["kind"] == q._lib.K_TILE)
    finally:
        q.qs_set_phase_tables(True)
    if kind == "brick":
        assert work[True] < 0.85 * work[False]


def test_phase_tables_survive_host_buffer_growth(q, orc):
    """Per-state resources of the table upload (device copy, pinned staging, event)
    stay valid across a reduction that grows the state's pinned result buffer: a
    fused apply with tables, a 12-qubit marginal (4096 results), a second fused
    apply, each against the oracle."""
    n = 14
    g = w.layered_u3_cz(n, 12, 4)
    ref1 = orc.run(n, g)
    ref2 = orc.apply_circuit(ref1.copy(), n, g)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    h = q.qs_alloc(n)
    try:
        q.qs_set_arith(h, q.ARITH_FIXED)
        q.qs_apply(h, g, None, p)
        assert np.max(np.abs(q.qs_get_state(h) - orc.as_complex(ref1))) < TOL
        qs12 = list(range(12))
        assert np.max(np.abs(q.qs_probs(h, qs12) - orc.marginal(ref1, n, qs12))) < 1e-12
        q.qs_apply(h, g, None, p)
        assert np.max(np.abs(q.qs_get_state(h) - orc.as_complex(ref2))) < TOL
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)


@pytest.mark.parametrize("n,kind", [(9, "brick"), (14, "brick"), (12, "rand"), (13, "hea")])
def test_rotation_pairs_match_oracle(q, orc, n, kind):
    """Q60 tile passes with groups of real rotations: four on one component of 16
    amplitudes as eight complex products, triples on octets as four and pairs on
    quads as two (with and without the preceding phase table fused into the
    group), against the oracle (1e-12) and with the switch off; groups of four
    take no more limb products than triples, triples no more than pairs, and
    pairs fewer than the rotations one at a time."""
    g = {"brick": lambda: w.layered_u3_cz(n, 12, 4), "rand": lambda: w.random_circuit(n, 400, 12),
         "hea": lambda: w.hea_ansatz(n, 4)[0]}[kind]()
    params = w.uniform_angles(400, 5)
    ref = orc.as_complex(orc.run(n, g, params))
    work = {}
    try:
        for on in (1, 4, 3, 2, 0):
            q.qs_set_rotation_pairs(on)
            p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
            h = q.qs_alloc(n)
            try:
                q.qs_set_arith(h, q.ARITH_FIXED)
                q.qs_timing_enable(h, True)
                q.qs_apply(h, g, params, p)
                recs = q.qs_timing_fetch(h)
                got = q.qs_get_state(h)
            finally:
                q.qs_free(h)
                q.qs_plan_free(p)
            assert np.max(np.abs(got - ref)) < TOL, on
            work[on] = sum(r["int_ops"] for r in recs if r["kind"] == q._lib.K_TILE)
    finally:
        q.qs_set_rotation_pairs(True)
    assert work[1] <= work[4] <= work[3] == work[2] < work[0]


def test_q60_buffer_between_tile_and_gate_passes(q, orc):
    """Consecutive Q60 tile passes keep Q60 integers in the state buffer; a
    per-gate pass after a tile pass, and the end of the call, find complex128
    again.  Plans of 4-qubit tiles on random circuits mix the two pass kinds
    (tile, gate, tile, ... and a trailing run of gate passes); each is checked
    to contain such a pattern and then against the oracle."""
    n = 14
    seen = set()
    for seed in range(5):
        g = w.random_circuit(n, 120, seed, two_qubit_prob=0.4)
        p = q.qs_plan_create_variant(n, g, 4, 0)
        kinds = "".join(str(k) for k, _, _ in q.qs_plan_passes(p))
        if "101" in kinds:
            seen.add("tile-gate-tile")
        if "110" in kinds:
            seen.add("tiles then gate")
        if kinds.endswith("1"):
            seen.add("ends on a tile pass")
        h = q.qs_alloc(n)
        try:
            q.qs_set_arith(h, q.ARITH_FIXED)
            q.qs_apply(h, g, None, p)
            psi = q.qs_get_state(h)
            # the buffer itself (not a converted copy) holds complex128 after the call
            assert abs(float(np.sum(np.abs(psi) ** 2)) - 1.0) < 1e-12
        finally:
            q.qs_free(h)
            q.qs_plan_free(p)
        assert np.max(np.abs(psi - orc.as_complex(orc.run(n, g)))) < TOL, (seed, kinds)
    assert {"tile-gate-tile", "tiles then gate", "ends on a tile pass"} <= seen, seen
