"""The learned fusion cost model: the GPU perceptron kernels against the CPU
oracle (forward, loss and every weight's gradient), training on the GPU, and
the learned planner against the greedy planner on circuits it was not trained
on -- both the amplitudes (oracle parity) and the measured time."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available()
    import paper_2212_14201_gb300 as q
    q.build()
    return q


@pytest.mark.parametrize("F,H,B", [(1, 1, 1), (3, 7, 13), (10, 32, 200)])
def test_mlp_kernels_match_oracle(q, orc, F, H, B):
    rng = np.random.Generator(np.random.PCG64(F * 100 + H))
    nw = orc.mlp_nweights(F, H)
    wts = rng.normal(size=nw) * 0.5
    x = rng.normal(size=(B, F))
    t = rng.normal(size=B)
    m = q.qs_mlp_create(F, H, wts)
    try:
        assert q.qs_mlp_num_weights(m) == nw
        assert np.array_equal(q.qs_mlp_get_weights(m), wts)
        y = q.qs_mlp_forward(m, x)
        assert np.max(np.abs(y - orc.mlp_forward(F, H, wts, x))) < 1e-12
        loss, g = q.qs_mlp_loss_grad(m, x, t)
        l0, g0 = orc.mlp_loss_grad(F, H, wts, x, t)
        assert abs(loss - l0) <= 1e-12 * max(1.0, abs(l0))
        assert np.max(np.abs(g - g0)) <= 1e-12 * max(1.0, np.max(np.abs(g0)))
    finally:
        q.qs_mlp_free(m)


def test_mlp_training_fits_a_smooth_function(q):
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.uniform(-1, 1, size=(256, 4))
    t = np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] - 0.3 * x[:, 3]
    m = q.qs_mlp_create(4, 16, None, 11)
    try:
        l0, _ = q.qs_mlp_loss_grad(m, x, t)
        loss = q.qs_mlp_train(m, x, t, 3000, 1e-2)
        assert loss < 0.02 * l0
    finally:
        q.qs_mlp_free(m)


def test_learned_plan_versus_greedy(q, orc):
    """Train on per-pass timings of n=20..22 random circuits (seeds 100..; passes of
    every candidate kind: widths 10..12, both ways of choosing a pass's qubits, and
    plain per-gate kernels), then on held-out circuits: the learned plan gives the
    oracle's amplitudes, every pass is a valid reordering, and the judge holds: the
    learned plan is never measurably slower than the greedy plan.  The measured
    ratio is printed (on these families the greedy choices are already the best
    ones the planner can make, and the learned plan keeps them)."""
    import torch
    from paper_2212_14201_gb300 import costmodel
    train_c = [(n, w.random_circuit(n, 300, 100 + i, two_qubit_prob=0.4), None) for i, n in enumerate((20, 21, 22, 22))]
    X, t = costmodel.collect(train_c, repeats=2, stream=torch.cuda.current_stream())
    assert X.shape[1] == q._lib.PASS_FEATURES and len(t) > 50
    m, loss = costmodel.train(X, t, epochs=3000)
    try:
        assert np.isfinite(loss)
        for n, seed in ((18, 300), (22, 301)):
            g = w.random_circuit(n, 400, seed, two_qubit_prob=0.4)
            pl = q.qs_plan_create_learned(n, g, m)
            pg = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
            order = np.concatenate([idx for _, _, idx in q.qs_plan_passes(pl)])
            assert sorted(order.tolist()) == list(range(len(g)))
            h = q.qs_alloc(n, torch.cuda.current_stream())
            try:
                if n <= 18:
                    q.qs_apply(h, g, None, pl)
                    assert np.max(np.abs(q.qs_get_state(h) - orc.as_complex(orc.run(n, g)))) < 1e-12
                times = {}
                for name, p in (("learned", pl), ("greedy", pg)):
                    q.qs_apply(h, g, None, p)
                    torch.cuda.synchronize()
                    best = 1e30
                    for _ in range(3):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        q.qs_apply(h, g, None, p)
                        e1.record()
                        torch.cuda.synchronize()
                        best = min(best, e0.elapsed_time(e1))
                    times[name] = best
                st = q.qs_plan_get_stats(pl)
                print(f"n={n}: learned {times['learned']:.3f} ms ({st['n_passes']} passes, greedy kept: "
                      f"{bool(st['learned_fallback'])}), greedy {times['greedy']:.3f} ms, "
                      f"gain {times['greedy'] / times['learned']:.4f}")
                assert times["learned"] <= 1.02 * times["greedy"] + 0.02
            finally:
                q.qs_free(h)
                q.qs_plan_free(pl)
                q.qs_plan_free(pg)
    finally:
        q.qs_mlp_free(m)


@pytest.mark.parametrize("n,kind,seed", [(28, "random", 300), (26, "layered", 303)])
def test_shipped_model_gains_over_greedy(q, orc, n, kind, seed):
    """The shipped cost model (trained on per-pass timings at n=24..30, seeds
    100..111) plans held-out circuits -- 600 random gates with 40 % two-qubit gates
    at n=28, a 16-layer U3 + CZ brickwork at n=26 -- faster than the greedy planner,
    measured: the gain (best of three applies each) must exceed both 2 % and three
    times the run-to-run spread of the greedy plan's own time (two independent
    best-of-three measurements).  The learned plan's amplitudes match the oracle
    (n=26) or the greedy plan's (n=28) within 1e-12."""
    import torch
    from paper_2212_14201_gb300 import costmodel
    g = w.random_circuit(n, 600, seed, two_qubit_prob=0.4) if kind == "random" else w.layered_u3_cz(n, 16, seed)
    model = costmodel.load()
    assert model is not None
    stream = torch.cuda.current_stream()
    pl = q.qs_plan_create_learned(n, g, model)
    pg = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    h = q.qs_alloc(n, stream)
    try:
        assert q.qs_plan_get_stats(pl)["learned_fallback"] == 0

        def best_of(p, reps=3):
            best = 1e30
            for _ in range(reps):
                q.qs_set_zero(h)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                q.qs_apply(h, g, None, p)
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            return best

        q.qs_set_zero(h)
        q.qs_apply(h, g, None, pl)  # warm-up
        t_greedy = best_of(pg)
        t_learned = best_of(pl)
        t_greedy2 = best_of(pg)
        spread = abs(t_greedy - t_greedy2) / min(t_greedy, t_greedy2)
        gain = min(t_greedy, t_greedy2) / t_learned
        print(f"n={n} {kind}: greedy {min(t_greedy, t_greedy2):.2f} ms ({q.qs_plan_get_stats(pg)['n_passes']} passes), "
              f"learned {t_learned:.2f} ms ({q.qs_plan_get_stats(pl)['n_passes']} passes), gain {gain:.4f}, "
              f"spread {spread:.4f}")
        assert gain > 1.0 + max(0.02, 3.0 * spread)
        q.qs_set_zero(h)
        q.qs_apply(h, g, None, pl)
        got = q.qs_get_state(h)
        if kind == "layered":
            want = orc.as_complex(orc.run(n, g))
        else:
            q.qs_set_zero(h)
            q.qs_apply(h, g, None, pg)
            want = q.qs_get_state(h)
        assert np.max(np.abs(got - want)) < 1e-12
    finally:
        q.qs_free(h)
        q.qs_plan_free(pl)
        q.qs_plan_free(pg)
        q.qs_mlp_free(model)


def test_config2_n32_plans_agree_with_plain_apply(q):
    """n=32 (64 GiB), 2000 random gates (40 % two-qubit, seed 2), the cost-model
    workload at full size: the oracle cannot hold this state, so the greedy plan
    and the learned plan (the shipped weights) are checked against plain per-gate
    apply, an independent code path: norm, <Z_i> for all 32 qubits and 2^16
    sampled amplitudes, each within 1e-12."""
    import torch
    from paper_2212_14201_gb300 import costmodel
    n = 32
    g = w.random_circuit(n, 2000, 2, two_qubit_prob=0.4)
    model = costmodel.load()
    plans = {"greedy": q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)}
    if model is not None:
        plans["learned"] = q.qs_plan_create_learned(n, g, model)
    idx = torch.randint(0, 1 << n, (1 << 16,), device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    h = q.qs_alloc(n, torch.cuda.current_stream())
    try:
        def run(p):
            q.qs_set_zero(h)
            q.qs_apply(h, g, None, p)
            norm2 = float(q.qs_probs(h, [])[0])
            ez = q.qs_expect_z_all(h)
            amps = torch.empty(2 << n, dtype=torch.float64, device="cuda")
            q.qs_get_state(h, amps)
            picked = amps.view(torch.complex128)[idx].clone()
            del amps
            torch.cuda.empty_cache()
            return norm2, ez, picked
        n0, ez0, a0 = run(None)
        assert abs(n0 - 1.0) < 1e-12
        for name, p in plans.items():
            n1, ez1, a1 = run(p)
            assert abs(n1 - 1.0) < 1e-12, name
            assert float(np.max(np.abs(ez1 - ez0))) < 1e-12, name
            assert float((a1 - a0).abs().max()) < 1e-12, name
    finally:
        q.qs_free(h)
        for p in plans.values():
            q.qs_plan_free(p)
        if model is not None:
            q.qs_mlp_free(model)
