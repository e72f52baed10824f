"""Pins of the oracle's partial-amplitude method (PartialAmpQVM, Section
"Multi-simulation methods": cut the two-qubit gates across a bisection into sums
of products and simulate the two halves per path): the amplitudes equal those of
the full state vector (the pinned plain simulator), GHZ by a chain crossing the
split, the path count, and a product circuit."""
import math

import numpy as np

import workloads as w

G = w.gate


def controlled_mix(n, count, seed):
    """Random gates plus multi-controlled rotations whose controls straddle any split."""
    rng = w.SplitMix64(seed)
    recs = list(w.random_circuit(n, count, seed))
    for _ in range(count // 5):
        t = rng.below(n)
        others = [q for q in range(n) if q != t]
        c1 = others[rng.below(len(others))]
        c2 = others[rng.below(len(others))]
        recs.append(G("RX", t, theta=rng.angle(), ctrl_mask=(1 << c1) | (1 << c2)))
        recs.append(G("CR", c1, t, theta=rng.angle()))
    return w.pack(recs)


def test_equals_full_state(orc):
    cases = [(5, controlled_mix(5, 20, 1)), (8, controlled_mix(8, 15, 2)), (10, w.layered_u3_cz(10, 6, 3))]
    for n, g in cases:
        full = orc.as_complex(orc.run(n, g))
        for n_low in range(1, n):
            amps, paths = orc.partial_amplitudes(n, g, n_low, np.arange(1 << n))
            assert np.max(np.abs(amps - full)) < 1e-13, (n, n_low)
            cut = sum(1 for r in g if _crosses(r, n_low))
            assert paths == 1 << cut


def _crosses(r, n_low):
    qs = {int(r["q0"])} | ({int(r["q1"])} if r["q1"] >= 0 else set())
    qs |= {b for b in range(64) if (int(r["ctrl_mask"]) >> b) & 1}
    return min(qs) < n_low <= max(qs)


def test_ghz_across_the_split(orc):
    n = 10
    g = w.pack([G("H", 0)] + [G("CNOT", i, i + 1) for i in range(n - 1)])
    amps, paths = orc.partial_amplitudes(n, g, 5, np.arange(1 << n))
    want = np.zeros(1 << n)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert paths == 2 and np.max(np.abs(amps - want)) < 1e-15


def test_product_circuit_and_subsets(orc):
    n, n_low = 9, 4
    lo = w.random_circuit(n_low, 50, 4)
    hi = w.random_circuit(n - n_low, 50, 5)
    hi_shift = hi.copy()
    hi_shift["q0"] += n_low
    hi_shift["q1"] = np.where(hi["q1"] >= 0, hi["q1"] + n_low, -1)
    g = np.concatenate([lo, hi_shift])
    want = np.kron(orc.as_complex(orc.run(n - n_low, hi)), orc.as_complex(orc.run(n_low, lo)))
    idx = np.array([0, 7, 511, 256, 300, 5], dtype=np.uint64)
    amps, paths = orc.partial_amplitudes(n, g, n_low, idx)
    assert paths == 1 and np.max(np.abs(amps - want[idx.astype(np.int64)])) < 1e-15
