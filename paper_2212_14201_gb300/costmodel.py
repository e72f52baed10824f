"""Learned fusion cost model.

The library's greedy planner takes each pass's qubits in program order at a fixed
tile width (12 qubits) and decides tile pass against per-gate kernels by a fixed
rule.  The learned planner (qs_plan_create_learned) lets a small perceptron
(qs_mlp_*) make those choices pass by pass: it predicts the log(milliseconds) of
candidate passes (widths 11 and 12; the greedy qubit set, a seeded one, and the
greedy set kept off one of its qubits; as one tile pass or gate by gate) and of
the greedy pass that would follow each, from their features
(qs_plan_features: the gates, and the kernel ops the tile engine would run for
the pass), and takes the candidate with the least predicted time per unit of
work over the two; the greedy plan is the fallback and the judge.  The network is trained on the GPU by the library's own
kernels (qs_mlp_train) from per-pass timings the library's kernel log records
(qs_timing_fetch), on the kinds of passes the planner chooses among.

Usage on a GPU machine:  python -m paper_2212_14201_gb300.costmodel --out FILE
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

from . import _lib

FEATURES = _lib.PASS_FEATURES
HIDDEN = 32
WEIGHTS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_weights.json")

_GATE_KINDS = (_lib.K_PHASE1, _lib.K_DIAG, _lib.K_ANTI, _lib.K_REAL, _lib.K_GENERAL)


def pass_timings(h: int, n: int, gates, plan: int, params=None, repeats: int = 2):
    """(features, ms) of every pass of `plan` that launched a kernel, measured on
    state `h` (n qubits) from the library's per-kernel event log."""
    feats = _lib.qs_plan_features(plan, gates)
    passes = _lib.qs_plan_passes(plan)
    _lib.qs_apply(h, gates, params, plan)      # warm-up
    _lib.qs_timing_enable(h, True)
    _lib.qs_timing_fetch(h)
    acc = np.zeros(len(passes))
    hit = np.zeros(len(passes), dtype=bool)
    for _ in range(repeats):
        _lib.qs_set_zero(h)
        _lib.qs_timing_fetch(h)
        _lib.qs_apply(h, gates, params, plan)
        recs = _lib.qs_timing_fetch(h)
        r = 0
        for i, (kind, qm, _) in enumerate(passes):
            if r >= len(recs):
                break
            rec = recs[r]
            ok = (rec["kind"] == _lib.K_TILE and rec["qubit_mask"] == qm) if kind == 1 else \
                 (rec["kind"] in _GATE_KINDS and rec["qubit_mask"] == qm)
            if ok:
                acc[i] += rec["ms"]
                hit[i] = True
                r += 1
    _lib.qs_timing_enable(h, False)
    return feats[hit], acc[hit] / repeats


def collect(circuits, tile_widths=(10, 11, 12), strategies=(0, 1, 2), plain: bool = True, repeats: int = 2,
            stream=None):
    """Timing data set over `circuits` = [(n, gates, params or None), ...]: the passes
    of plans of every width and strategy (qs_plan_create_variant), and with
    plain=True every gate of the plain per-gate plan."""
    X, y = [], []
    states = {}
    try:
        for n, gates, params in circuits:
            if n not in states:
                states[n] = _lib.qs_alloc(n, stream)
            plans = []
            for m in tile_widths:
                if m > n:
                    continue
                for st in strategies:
                    plans.append(_lib.qs_plan_create_variant(n, gates, m, st))
            if plain:
                plans.append(_lib.qs_plan_create(n, gates, _lib.PLAN_PLAIN, 1))
            for p in plans:
                try:
                    f, ms = pass_timings(states[n], n, gates, p, params, repeats)
                finally:
                    _lib.qs_plan_free(p)
                X.append(f)
                y.append(ms)
    finally:
        for h in states.values():
            _lib.qs_free(h)
    X = np.concatenate(X)
    y = np.concatenate(y)
    keep = y > 0
    return X[keep], np.log(y[keep])


def train(X, t, hidden: int = HIDDEN, epochs: int = 4000, lr: float = 3e-3, seed: int = 7):
    """Model handle trained on (X, log ms) by the GPU kernels; returns (handle, loss)."""
    m = _lib.qs_mlp_create(X.shape[1], hidden, None, seed)
    loss = _lib.qs_mlp_train(m, X, t, epochs, lr)
    return m, loss


def save(m: int, path: str = WEIGHTS_FILE, meta: dict | None = None, hidden: int = HIDDEN):
    w = _lib.qs_mlp_get_weights(m)
    with open(path, "w") as f:
        json.dump({"features": FEATURES, "hidden": hidden, "weights": w.tolist(), "meta": meta or {}}, f)


def load(path: str = WEIGHTS_FILE) -> int | None:
    """Model handle from a saved weight file, or None if there is none."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    return _lib.qs_mlp_create(d["features"], d["hidden"], np.asarray(d["weights"], dtype=np.float64), 0)


def default_training_circuits(ns=(24, 26, 28, 30), per_n: int = 2, seed0: int = 100):
    """Random circuits of the n=32 workload's mix (40 % two-qubit gates) at
    smaller n, seeds 100.., plus a layered U3 + CZ circuit per n (12 layers: deep
    enough for lookahead passes that span several layers)."""
    import workloads as w
    out = []
    s = seed0
    for n in ns:
        for _ in range(per_n):
            out.append((n, w.random_circuit(n, 400, s, two_qubit_prob=0.4), None))
            s += 1
        out.append((n, w.layered_u3_cz(n, 12, s), None))
        s += 1
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS_FILE)
    ap.add_argument("--ns", default="24,26,28,30")
    ap.add_argument("--per-n", type=int, default=2)
    ap.add_argument("--epochs", type=int, default=6000)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    circuits = default_training_circuits(tuple(int(x) for x in args.ns.split(",")), args.per_n)
    X, t = collect(circuits, stream=torch.cuda.current_stream())
    m, loss = train(X, t, epochs=args.epochs)
    save(m, args.out, {"samples": int(len(t)), "loss": loss, "ns": args.ns, "per_n": args.per_n})
    print(json.dumps({"samples": int(len(t)), "loss": loss, "out": args.out}))
    _lib.qs_mlp_free(m)


if __name__ == "__main__":
    main()
