"""The complex64 variant (qs_alloc_c64): FP32 gate arithmetic in the per-gate and
tile-pass kernels, reductions and the canonical sampler on the stored values
widened to double.

Tolerances follow from the arithmetic.  With u = 2^-24 (float rounding), one 2x2
op on an amplitude pair changes the state by at most about 8 u in 2-norm (matrix
entries rounded to float, at most four fused products per component).  Ops act
unitarily on earlier errors, so G ops stay within 8 G u of the exact state.
Reductions of a stored complex64 state are compared with the oracle on the same
values widened to double: 1e-12, as for complex128."""
import math

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available()
    import paper_2212_14201_gb300 as q
    q.build()
    return q


def c64_run(q, n, gates, fused, params=None):
    h = q.qs_alloc_c64(n)
    p = q.qs_plan_create(n, gates, q.PLAN_GREEDY, 5) if fused else None
    try:
        assert q.qs_state_precision(h) == 64
        q.qs_apply(h, gates, params, p)
        return q.qs_get_state(h)
    finally:
        q.qs_free(h)
        if p:
            q.qs_plan_free(p)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("n,ng,seed", [(1, 30, 0), (3, 80, 1), (7, 200, 2), (12, 200, 0), (14, 400, 5)])
def test_circuits_against_oracle(q, orc, n, ng, seed, fused):
    g = w.random_circuit(n, ng, seed)
    got = c64_run(q, n, g, fused).astype(np.complex128)
    ref = orc.as_complex(orc.run(n, g))
    err = float(np.linalg.norm(got - ref))
    assert err <= 8 * ng * U32, err
    assert abs(float(np.vdot(got, got).real) - 1.0) <= 16 * ng * U32


def test_stored_state_reductions_and_sampling(q, orc):
    """On the stored complex64 state widened to double: probabilities, marginals,
    <Z_i>, a Pauli sum (1e-12) and the canonical sampler (bit-exact)."""
    n = 13
    g = w.random_circuit(n, 300, 7)
    terms = w.random_paulis(n, 12, 3)
    h = q.qs_alloc_c64(n)
    try:
        q.qs_apply(h, g, None, None)
        st = q.qs_get_state(h).astype(np.complex128)
        ref = st.view(np.float64)
        assert np.max(np.abs(q.qs_probs(h, list(range(n))) - orc.probs(ref, n))) < 1e-12
        for qs_ in ([], [0], [5, 2, 11], list(range(10)), list(range(12))):
            assert np.max(np.abs(q.qs_probs(h, qs_) - orc.marginal(ref, n, qs_))) < 1e-12
        assert np.max(np.abs(q.qs_expect_z_all(h) - orc.expect_z(ref, n))) < 1e-12
        assert abs(q.qs_expect_pauli(h, terms) - orc.expect_pauli(ref, n, terms)) < 1e-12
        assert np.array_equal(q.qs_sample(h, 21, 20000), orc.sample(ref, n, 21, 20000))
    finally:
        q.qs_free(h)


def test_measure_and_program(q, orc):
    n = 9
    g = w.random_circuit(n, 120, 4)
    h = q.qs_alloc_c64(n)
    try:
        q.qs_apply(h, g, None, None)
        st = q.qs_get_state(h).astype(np.complex128)
        for qubit, u in ((0, 0.3), (4, 0.7), (8, 0.1)):
            o, p1 = q.qs_measure(h, qubit, u)
            oo, pp1, post = orc.measure(st, n, qubit, u)
            assert abs(p1 - pp1) < 1e-12 and o == oo
            got = q.qs_get_state(h).astype(np.complex128)
            # the kept part is scaled in double and rounded once to float
            assert np.max(np.abs(got - orc.as_complex(post))) <= 2 * U32 * np.max(np.abs(orc.as_complex(post)))
            st = got
        prog, gates = w.random_program(n, 3)
        q.qs_set_zero(h)
        cb, rec = q.qs_run_program(h, prog, gates, seed=9)
        _, cb0, rec0 = orc.run_program(n, prog, gates, seed=9)
        if np.array_equal(cb, cb0):
            assert np.max(np.abs(rec - rec0)) < 1e-4
    finally:
        q.qs_free(h)


def test_roundtrip_and_unsupported(q):
    import torch
    n = 6
    h = q.qs_alloc_c64(n)
    try:
        v = (np.arange(1 << n) + 1j * np.arange(1 << n)[::-1]).astype(np.complex64)
        q.qs_set_state(h, v)
        assert np.array_equal(q.qs_get_state(h), v)
        t = torch.empty(2 << n, dtype=torch.float32, device="cuda")
        q.qs_get_state(h, t)
        assert np.array_equal(t.cpu().numpy().view(np.complex64), v)
        with pytest.raises(ValueError):
            q.qs_set_state(h, v.astype(np.complex128))   # wrong element size
        with pytest.raises(q.QsimError):
            q.qs_apply_matrix(h, [0], np.eye(2))
        with pytest.raises(q.QsimError):
            q.qs_set_arith(h, q.ARITH_FIXED)
        g, npar = w.hea_ansatz(n, 1)
        with pytest.raises(q.QsimError):
            q.qs_adjoint_grad(h, g, w.uniform_angles(npar, 1), w.zz_chain(n))
    finally:
        q.qs_free(h)


def test_full_size_against_complex128(q):
    """n=30 brickwork (890 gates), complex64 fused against complex128 fused on
    65536 sampled amplitudes and through the norm."""
    import torch
    n = 30
    g = w.layered_u3_cz(n, 20, 1)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    idx = torch.randint(0, 1 << n, (1 << 16,), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    h = q.qs_alloc(n)
    try:
        q.qs_apply(h, g, None, p)
        amps = torch.empty(2 << n, dtype=torch.float64, device="cuda")
        q.qs_get_state(h, amps)
        ref = amps.view(torch.complex128)[idx].clone()
        del amps
    finally:
        q.qs_free(h)
    torch.cuda.empty_cache()
    h = q.qs_alloc_c64(n)
    try:
        q.qs_apply(h, g, None, p)
        assert abs(q.qs_probs(h, [])[0] - 1.0) <= 16 * len(g) * U32
        amps = torch.empty(2 << n, dtype=torch.float32, device="cuda")
        q.qs_get_state(h, amps)
        got = amps.view(torch.complex64)[idx].to(torch.complex128)
        # the whole-state bound 8 G u caps every amplitude's error
        assert float((got - ref).abs().max()) <= 8 * len(g) * U32
        del amps
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)
