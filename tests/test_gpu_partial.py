"""GPU parity of partial amplitudes (qs_partial_amplitudes) against the CPU
oracle's cut-and-sum computation and the full state vector (1e-12), for every
split point of small circuits, multi-controlled cuts and fused / per-gate block
runs; at n=30 against the full-state GPU simulation; at n=40 (no full state)
between two different split points."""
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


def controlled_mix(n, count, seed):
    rng = w.SplitMix64(seed)
    recs = list(w.random_circuit(n, count, seed))
    for _ in range(count // 5):
        t = rng.below(n)
        others = [x for x in range(n) if x != t]
        c1, c2 = others[rng.below(len(others))], others[rng.below(len(others))]
        recs.append(G("RX", t, theta=rng.angle(), ctrl_mask=(1 << c1) | (1 << c2)))
        recs.append(G("CR", c1, t, theta=rng.angle(), dagger=rng.below(2)))
    return w.pack(recs)


@pytest.mark.parametrize("fuse", [False, True])
def test_small_circuits_every_split(q, orc, fuse):
    for n, g in ((5, controlled_mix(5, 20, 1)), (8, controlled_mix(8, 15, 2)), (12, w.layered_u3_cz(12, 8, 3))):
        full = orc.as_complex(orc.run(n, g))
        idx = np.arange(1 << n, dtype=np.uint64)
        for n_low in range(1, n):
            amps, paths = q.qs_partial_amplitudes(n, g, n_low, idx, fuse=fuse)
            ref, opaths = orc.partial_amplitudes(n, g, n_low, idx)
            assert paths == opaths
            assert np.max(np.abs(amps - ref)) < TOL and np.max(np.abs(amps - full)) < TOL, (n, n_low)


def test_parametrised_and_subset(q, orc):
    n = 10
    g, npar = w.hea_ansatz(n, 3)
    th = w.uniform_angles(npar, 6)
    idx = np.array([0, 5, 1023, 512, 77, 77, 300], dtype=np.uint64)
    amps, _ = q.qs_partial_amplitudes(n, g, 4, idx, params=th)
    full = orc.as_complex(orc.run(n, g, th))
    assert np.max(np.abs(amps - full[idx.astype(np.int64)])) < TOL


def test_full_size_against_full_state(q):
    """n=30 brickwork (depth 8): 4096 sampled amplitudes by cutting at 15 against
    the full-state fused simulation."""
    import torch
    n = 30
    g = w.layered_u3_cz(n, 8, 1)
    rng = np.random.Generator(np.random.PCG64(1))
    idx = rng.integers(0, 1 << n, 4096, dtype=np.uint64)
    amps, paths = q.qs_partial_amplitudes(n, g, 15, idx)
    assert paths == 1 << 4   # the CZ on (14, 15) of each of the 4 even layers is cut
    h = q.qs_alloc(n)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    try:
        q.qs_apply(h, g, None, p)
        t = torch.empty(2 << n, dtype=torch.float64, device="cuda")
        q.qs_get_state(h, t)
        full = t.view(torch.complex128)[torch.tensor(idx.astype(np.int64), device="cuda")].cpu().numpy()
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)
    assert np.max(np.abs(amps - full)) < TOL


def test_beyond_one_state(q):
    """n=40 (a 16 TiB state): the same amplitudes from two different cuts."""
    n = 40
    g = w.layered_u3_cz(n, 6, 2)
    rng = np.random.Generator(np.random.PCG64(2))
    idx = rng.integers(0, 1 << n, 2000, dtype=np.uint64)
    a, pa = q.qs_partial_amplitudes(n, g, 20, idx)
    b, pb = q.qs_partial_amplitudes(n, g, 22, idx)
    assert pa == 8 and pb == 8
    assert np.max(np.abs(a - b)) < TOL
    assert 0 < np.sum(np.abs(a) ** 2) * (1 << n) / len(idx) < 10   # mean |amp|^2 ~ 2^-n


def test_errors(q):
    g = w.pack([G("H", 0)])
    for n, n_low in ((1, 0), (4, 0), (4, 4), (80, 40)):
        with pytest.raises(q.QsimError):
            q.qs_partial_amplitudes(n, g, n_low, [0])
    with pytest.raises(q.QsimError):
        q.qs_partial_amplitudes(4, g, 2, [16])
