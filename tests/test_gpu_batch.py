"""GPU parity of the batched persistent variational evaluation (qs_batch_*):
every set's energy and gradient against the CPU oracle's adjoint recursion on
small sets, and against the single-state GPU adjoint kernel (an independent code
path) for the full 1024-set workload.  Energies within 1e-12; every gradient
entry within 1e-9 relative, plus the derived rounding floor of tests/_tol.py for
entries that vanish."""
import numpy as np
import pytest

import workloads as w
from tests._tol import grad_close, grad_report, h1_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available()
    import paper_2212_14201_gb300 as q
    q.build()
    return q


def rel_close(a, b, n, gates, terms):
    """Element-wise: |a - b| <= 1e-9 |b| + floor(n, G, ||H||_1)."""
    ok = grad_close(a, b, n, len(gates), h1_of(terms))
    if not ok:
        print(grad_report(a, b, n, len(gates), h1_of(terms)))
    return ok


def make_sets(ns, layers, seed, ham="tfim"):
    gl, npl, tl = [], [], []
    for n in ns:
        g, npar = w.hea_ansatz(int(n), layers)
        gl.append(g)
        npl.append(npar)
        tl.append(w.tfim(int(n), 0.7) if ham == "tfim" else w.random_paulis(int(n), 8, seed + int(n)))
    params = w.uniform_angles(int(sum(npl)), seed)
    return gl, npl, tl, params


def split(params, npl):
    out, o = [], 0
    for k in npl:
        out.append(params[o:o + k])
        o += k
    return out


@pytest.mark.parametrize("ham", ["tfim", "rand"])
def test_batch_matches_oracle(q, orc, ham):
    ns = [1, 2, 3, 5, 8, 11, 12, 13, 14, 6, 9, 10]
    gl, npl, tl, params = make_sets(ns, 3, 7, ham)
    b = q.qs_batch_create(ns, gl, npl, tl)
    try:
        e = np.empty(len(ns))
        g = np.empty(len(params))
        q.qs_batch_run(b, params, e, g)
    finally:
        q.qs_batch_free(b)
    for s, (n, gates, terms, th, gs) in enumerate(zip(ns, gl, tl, split(params, npl), split(g, npl))):
        e0, g0 = orc.adjoint_grad(n, gates, th, terms)
        assert abs(e[s] - e0) < 1e-12, s
        assert rel_close(gs, g0, n, gates, terms), s


@pytest.mark.parametrize("ctas", [0, 1, 2, 4, 8])
def test_cluster_and_single_cta_items_together(q, orc, ctas):
    """Sets with at least c tiles per pass are shared by a cluster of c CTAs
    (tiles split over the cluster, gradient partials summed across it); smaller
    sets run one per CTA.  Both kinds in one launch, for every cluster size,
    against the oracle, and bit-identical on a rerun."""
    ns = [17, 10, 15, 14, 12, 16, 13, 11, 14, 9]
    gl, npl, tl, params = make_sets(ns, 3, 21, "rand")
    q.qs_set_batch_cluster(ctas)
    try:
        b = q.qs_batch_create(ns, gl, npl, tl)
    finally:
        q.qs_set_batch_cluster(0)
    try:
        if ctas:
            assert q.qs_batch_cluster(b) == ctas
        outs = []
        for _ in range(2):
            e = np.empty(len(ns))
            g = np.empty(len(params))
            q.qs_batch_run(b, params, e, g)
            outs.append((e, g))
    finally:
        q.qs_batch_free(b)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    e, g = outs[0]
    for s, (n, gates, terms, th, gs) in enumerate(zip(ns, gl, tl, split(params, npl), split(g, npl))):
        e0, g0 = orc.adjoint_grad(n, gates, th, terms)
        assert abs(e[s] - e0) < 1e-12, s
        assert rel_close(gs, g0, n, gates, terms), s


def test_batch_general_records(q, orc):
    """Controls, dagger records, shared parameters, parametrised diagonal gates
    whose target falls outside a tile (n=16 > 11 tile qubits)."""
    sets = []
    for n, seed in ((16, 1), (13, 2), (7, 3)):
        rng = w.SplitMix64(seed)
        recs = [w.gate("H", qq) for qq in range(n)]
        for i in range(5 * n):
            t = rng.below(n)
            c = (t + 1 + rng.below(n - 1)) % n
            k = i % 6
            if k == 0:
                recs.append(w.gate("RZ", t, param_idx=rng.below(4)))
            elif k == 1:
                recs.append(w.gate("CR", c, t, param_idx=rng.below(4)))
            elif k == 2:
                recs.append(w.gate("RX", t, param_idx=rng.below(4), ctrl_mask=1 << c, dagger=i & 1))
            elif k == 3:
                recs.append(w.gate("CNOT", c, t))
            elif k == 4:
                recs.append(w.gate("U3", t, theta=rng.angle(), phi=rng.angle(), lam=rng.angle()))
            else:
                recs.append(w.gate("P", t, param_idx=rng.below(4), dagger=1))
        sets.append((n, w.pack(recs), 4, w.random_paulis(n, 6, seed)))
    ns = [s[0] for s in sets]
    params = w.uniform_angles(12, 5)
    b = q.qs_batch_create(ns, [s[1] for s in sets], [4, 4, 4], [s[3] for s in sets])
    try:
        e = np.empty(3)
        g = np.empty(12)
        q.qs_batch_run(b, params, e, g)
    finally:
        q.qs_batch_free(b)
    for i, (n, gates, _, terms) in enumerate(sets):
        e0, g0 = orc.adjoint_grad(n, gates, params[4 * i:4 * i + 4], terms)
        assert abs(e[i] - e0) < 1e-12
        assert rel_close(g[4 * i:4 * i + 4], g0, n, gates, terms)


def test_graph_replay_and_device_path(q, orc):
    import torch
    ns = [4, 9, 12, 3]
    gl, npl, tl, p1 = make_sets(ns, 2, 11)
    p2 = w.uniform_angles(len(p1), 12)
    b = q.qs_batch_create(ns, gl, npl, tl)
    try:
        outs = []
        for p in (p1, p2, p1):     # first call captures the graph, the others replay it
            e = np.empty(len(ns))
            g = np.empty(len(p))
            q.qs_batch_run(b, p, e, g)
            outs.append((e, g))
        assert np.array_equal(outs[0][0], outs[2][0]) and np.array_equal(outs[0][1], outs[2][1])
        for s, (n, gates, terms, th) in enumerate(zip(ns, gl, tl, split(p2, npl))):
            e0, g0 = orc.adjoint_grad(n, gates, th, terms)
            assert abs(outs[1][0][s] - e0) < 1e-12 and rel_close(split(outs[1][1], npl)[s], g0, n, gates, terms)
        pd = torch.tensor(p2, dtype=torch.float64, device="cuda")
        ed = torch.empty(len(ns), dtype=torch.float64, device="cuda")
        gd = torch.empty(len(p2), dtype=torch.float64, device="cuda")
        q.qs_batch_run(b, pd, ed, gd)
        assert np.array_equal(ed.cpu().numpy(), outs[1][0]) and np.array_equal(gd.cpu().numpy(), outs[1][1])
        assert q.qs_batch_last_ms(b) > 0
    finally:
        q.qs_batch_free(b)


def test_full_batch_matches_single_state_adjoint(q):
    """The batched workload at full size: 1024 sets, n uniform in 10..20, 8-layer
    RY/RZ + CNOT-ring ansatz, TFIM (h=0.7), angles uniform (seed 33).  Every set
    against the single-state adjoint kernel (qs_adjoint_grad)."""
    ns = w.batch_qubit_counts(1024, 3)
    gl, npl, tl, params = make_sets(ns, 8, 33)
    b = q.qs_batch_create(ns, gl, npl, tl)
    try:
        e = np.empty(len(ns))
        g = np.empty(len(params))
        q.qs_batch_run(b, params, e, g)
    finally:
        q.qs_batch_free(b)
    gs = split(g, npl)
    ths = split(params, npl)
    hs = {}
    try:
        for s in range(len(ns)):
            n = int(ns[s])
            if n not in hs:
                hs[n] = q.qs_alloc(n)
            e1, g1 = q.qs_adjoint_grad(hs[n], gl[s], ths[s], tl[s])
            assert abs(e[s] - e1) < 1e-11, s
            assert rel_close(gs[s], g1, n, gl[s], tl[s]), s
    finally:
        for h in hs.values():
            q.qs_free(h)


def test_batch_groups_and_fused_backward_steps(q, orc):
    """Sets built to exercise diagonal groups (Z and P generators, members with and
    without parameters, a parameter shared inside a group) and the one-sweep
    backward of real ops, against the oracle's adjoint recursion."""
    sets = [(n, *w.mixed_layers_circuit(n, 3, 20 + n)) for n in (4, 9, 13)]
    ns = [s[0] for s in sets]
    nps = [s[2] for s in sets]
    params = w.uniform_angles(int(sum(nps)), 21)
    terms = [w.random_paulis(n, 8, n) for n in ns]
    b = q.qs_batch_create(ns, [s[1] for s in sets], nps, terms)
    try:
        e = np.empty(len(ns))
        g = np.empty(len(params))
        q.qs_batch_run(b, params, e, g)
    finally:
        q.qs_batch_free(b)
    off = 0
    for i, (n, gates, npar) in enumerate(sets):
        e0, g0 = orc.adjoint_grad(n, gates, params[off:off + npar], terms[i])
        assert abs(e[i] - e0) < 1e-12
        assert rel_close(g[off:off + npar], g0, n, gates, terms[i])
        off += npar
