"""GPU parity of the adjoint gradient (qs_adjoint_grad and the torch.autograd
binding) against the CPU oracle's adjoint recursion, parameter shift and central
finite differences.  Every gradient entry within 1e-9 relative (plus the derived
rounding floor of tests/_tol.py for entries that vanish); energies within 1e-12."""
import math

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


def gpu_grad(q, n, g, th, H, arith=None):
    h = q.qs_alloc(n)
    try:
        if arith is not None:
            q.qs_set_arith(h, arith)
        return q.qs_adjoint_grad(h, g, th, H)
    finally:
        q.qs_free(h)


def rel_close(a, b, n, gates, terms):
    """Element-wise: |a - b| <= 1e-9 |b| + floor(n, G, ||H||_1)."""
    ok = grad_close(a, b, n, len(gates), h1_of(terms))
    if not ok:
        print(grad_report(a, b, n, len(gates), h1_of(terms)))
    return ok


@pytest.mark.parametrize("arith", ["fp64", "q60"])
@pytest.mark.parametrize("n,layers,ham", [(2, 2, "tfim"), (5, 3, "zz"), (9, 4, "tfim"), (12, 12, "zz"), (14, 3, "rand")])
def test_adjoint_matches_oracle(q, orc, arith, n, layers, ham):
    g, npar = w.hea_ansatz(n, layers)
    th = w.uniform_angles(npar, 4 + n)
    H = {"tfim": w.tfim(n, 0.7), "zz": w.zz_chain(n), "rand": w.random_paulis(n, 20, 3)}[ham]
    mode = {"fp64": q.ARITH_FP64, "q60": q.ARITH_FIXED}[arith]
    e, grad = gpu_grad(q, n, g, th, H, mode)
    e0, g0 = orc.adjoint_grad(n, g, th, H)
    assert abs(e - e0) < 1e-12
    assert rel_close(grad, g0, n, g, H)


def test_n12_against_parameter_shift_and_finite_differences(q, orc):
    """The n=12 check of the adjoint workload: 12-layer RY/RZ + CNOT-ring ansatz,
    ZZ chain; parameter shift (exact for these rotations) and central differences
    with h = 1e-6, both from the oracle."""
    n, layers = 12, 12
    g, npar = w.hea_ansatz(n, layers)
    th = w.uniform_angles(npar, 4)
    H = w.zz_chain(n)
    e, grad = gpu_grad(q, n, g, th, H)
    idx = list(range(0, npar, 23))[:12]
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += math.pi / 2
        tm[k] -= math.pi / 2
        shift = 0.5 * (orc.energy(n, g, tp, H) - orc.energy(n, g, tm, H))
        assert rel_close(grad[k:k + 1], [shift], n, g, H)
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (orc.energy(n, g, tp, H) - orc.energy(n, g, tm, H)) / (2 * h)
        assert abs(grad[k] - fd) < 1e-7


def test_controlled_daggered_and_shared_parameters(q, orc):
    n = 7
    recs = [w.gate("H", qq) for qq in range(n)]
    recs += [w.gate("RX", 1, param_idx=0, ctrl_mask=0b0000001), w.gate("CR", 2, 5, param_idx=1),
             w.gate("RY", 0, param_idx=2, dagger=1), w.gate("P", 6, param_idx=0),
             w.gate("RZ", 3, param_idx=3, ctrl_mask=0b1000000), w.gate("CNOT", 3, 1), w.gate("RX", 2, param_idx=2),
             w.gate("U3", 4, theta=0.3, phi=0.2, lam=0.1), w.gate("RY", 4, param_idx=1)]
    g = w.pack(recs)
    th = np.array([0.4, 1.3, -0.8, 2.2])
    H = w.random_paulis(n, 9, 2)
    e, grad = gpu_grad(q, n, g, th, H)
    e0, g0 = orc.adjoint_grad(n, g, th, H)
    assert abs(e - e0) < 1e-12 and rel_close(grad, g0, n, g, H)


def test_rejects_unsupported_parameter(q):
    g = w.pack([w.gate("U3", 0, param_idx=0)])
    h = q.qs_alloc(2)
    try:
        with pytest.raises(q.QsimError):
            q.qs_adjoint_grad(h, g, np.array([0.1]), w.zz_chain(2))
    finally:
        q.qs_free(h)


def test_torch_autograd_function(q, orc):
    import torch

    from paper_2212_14201_gb300.autograd import Expectation
    n = 8
    g, npar = w.hea_ansatz(n, 3)
    H = w.tfim(n, 0.7)
    th = torch.tensor(w.uniform_angles(npar, 9), dtype=torch.float64, requires_grad=True)
    f = Expectation(n, g, H)
    e = f(th)
    (2.0 * e).backward()
    e0, g0 = orc.adjoint_grad(n, g, th.detach().numpy(), H)
    assert abs(e.item() - e0) < 1e-12
    H2 = H.copy()
    H2["coef"] *= 2.0  # the loss is 2 E
    assert rel_close(th.grad.numpy(), 2.0 * g0, n, g, H2)
    f.close()


def test_full_size_adjoint_invariants(q):
    """n=28, 12 layers (1008 gates, 672 parameters), ZZ chain: the launch
    configuration of the adjoint benchmark.  Properties that hold at any size:
    the backward sweep returns the state to |0...0>, |E| <= 27, and the gradient
    of a parameter equals the parameter-shift difference of two GPU energies."""
    import torch
    n, layers = 28, 12
    g, npar = w.hea_ansatz(n, layers)
    th = w.uniform_angles(npar, 4)
    H = w.zz_chain(n)
    h = q.qs_alloc(n)
    try:
        e, grad = q.qs_adjoint_grad(h, g, th, H)
        assert abs(e) <= 27 + 1e-9 and np.all(np.isfinite(grad))
        back = torch.empty(2 << n, dtype=torch.float64, device="cuda")
        q.qs_get_state(h, back)
        z = back.view(torch.complex128)
        assert abs(z[0].item() - 1.0) < 1e-10
        z[0] = 0
        assert float(z.abs().max()) < 1e-10
        del back, z
        k = 100
        def energy(t):
            q.qs_set_zero(h)
            q.qs_apply(h, g, t)
            return q.qs_expect_pauli(h, H)
        tp, tm = th.copy(), th.copy()
        tp[k] += math.pi / 2
        tm[k] -= math.pi / 2
        shift = 0.5 * (energy(tp) - energy(tm))
        assert rel_close(grad[k:k + 1], [shift], n, g, H)
    finally:
        q.qs_free(h)


def test_config4_full_depth_against_oracle(q, orc):
    """The adjoint workload's circuit (12 layers of RY, RZ and the CNOT ring; ZZ
    chain) at the largest size the oracle's adjoint recursion finishes in about a
    minute, n=24 (864 gates, 576 parameters): energy within 1e-12 and every
    gradient entry within 1e-9 relative of the oracle's, fused backward (Q60)."""
    n, layers = 24, 12
    g, npar = w.hea_ansatz(n, layers)
    th = w.uniform_angles(npar, 4)
    H = w.zz_chain(n)
    e, grad = gpu_grad(q, n, g, th, H)
    e0, g0 = orc.adjoint_grad(n, g, th, H)
    print(f"n={n} energy err {abs(e - e0):.3e}; " + grad_report(grad, g0, n, len(g), h1_of(H)))
    assert abs(e - e0) < 1e-12
    assert rel_close(grad, g0, n, g, H)


@pytest.mark.parametrize("n,layers", [(9, 3), (13, 4)])
def test_per_gate_backward_path(q, orc, n, layers):
    """The gate-by-gate backward sweep (qs_set_adjoint_fused(0)) against the oracle."""
    g, npar = w.hea_ansatz(n, layers)
    th = w.uniform_angles(npar, 40 + n)
    H = w.tfim(n, 0.7)
    q.qs_set_adjoint_fused(False)
    try:
        e, grad = gpu_grad(q, n, g, th, H)
    finally:
        q.qs_set_adjoint_fused(True)
    e0, g0 = orc.adjoint_grad(n, g, th, H)
    assert abs(e - e0) < 1e-12 and rel_close(grad, g0, n, g, H)


@pytest.mark.parametrize("n,layers", [(3, 2), (8, 3), (13, 3)])
def test_fused_backward_groups_and_pairs(q, orc, n, layers):
    """Diagonal groups (Z and P generators, members with and without parameters,
    a parameter shared inside a group) and real pairs (Y generators, dagger flags,
    pairs without generators) against the oracle's adjoint recursion, fused
    backward (Q60) and the per-gate path (FP64)."""
    g, npar = w.mixed_layers_circuit(n, layers, 5 + n)
    th = w.uniform_angles(npar, 9 + n)
    H = w.random_paulis(n, 12, 4)
    e0, g0 = orc.adjoint_grad(n, g, th, H)
    for arith in (q.ARITH_FIXED, q.ARITH_FP64):
        e, grad = gpu_grad(q, n, g, th, H, arith)
        assert abs(e - e0) < 1e-12 and rel_close(grad, g0, n, g, H), arith
