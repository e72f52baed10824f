"""Benchmark of the full-amplitude hot path on the n=30 layered circuit.

Workload: n=30 complex128 state (16 GiB) from |0...0>, 20 layers of U3 (angles
uniform in [0, 2pi), seed 1) on every qubit followed by CZ on brickwork
neighbour pairs (even layers (2j,2j+1), odd layers (2j+1,2j+2)): 600 U3 + 290 CZ.
One step = reset to |0>, apply the circuit (fused plan; plain per-gate apply is
timed beside it), the squared norm, and 1e6 measurement samples (seed 11).
Metric: amp-updates/s = (gates x 2^n) / step time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (the state does not shard
without a collective; see the design notes) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

METRIC = "amp-updates/s & HBM GB/s (n=30, fused vs plain); batched VQE grad evals/s"
UNIT = "amp-updates/s"
SHOTS = 1_000_000
SAMPLE_SEED = 11
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak derived from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz.
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9
# Wide integer multiply-add peak (Q60 engine): a warp's mad.wide.s32 (32x32->64)
# holds the FMA-heavy pipe of its SM sub-partition for 4 cycles (ncu pipe counters
# of a register-only loop of them), so 152 SMs x 4 sub-partitions x 8 lanes/clk x
# 2.07 GHz.
INT_PEAK_OPS = 152 * 4 * 8 * 2.07e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=30, help="qubits (30 is the benchmark workload)")
    ap.add_argument("--depth", type=int, default=20)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-gate arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched / adjoint / n=32 side workloads")
    ap.add_argument("--no-n32", action="store_true", help="skip the n=32 learned-vs-greedy plan comparison")
    ap.add_argument("--only-batch", action="store_true",
                    help="profiling aid: run only the batched VQE workload and print its result")
    ap.add_argument("--batch-sets", type=int, default=1024, help="parameter sets of the batched VQE workload")
    ap.add_argument("--only-reductions", type=int, default=0, metavar="N",
                    help="profiling aid: run only the reduction timings on an N-qubit state and print them")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def whole_job_value(world: int, units_per_rank: float, ms_max: float) -> float:
    """Units all ranks processed (each rank runs the same replica) / the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def traffic_for(kernel_kind: int):
    """DRAM bytes per launch from a committed ncu summary, if its kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    ent = d.get(str(kernel_kind))
    if not ent:
        return None
    src = os.path.join(ROOT, ent["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if h != ent["sha256"]:
        return None
    return ent["bytes_per_launch_full"]


def roofline(records, hbm_peak_gbs):
    """Dominant kernel class by total device time; algorithmic bytes and flops per launch."""
    by = {}
    for r in records:
        d = by.setdefault(r["kind"], {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0, "iops": 0.0})
        d["ms"] += r["ms"]
        d["launches"] += 1
        rw = 1 if r["kind"] == 20 else 2   # reductions read only; gate kernels read and write
        d["bytes"] += r["items"] * 16.0 * rw
        d["flops"] += r["flops"]
        d["iops"] += r["int_ops"]
    kind, d = max(by.items(), key=lambda kv: kv[1]["ms"])
    per_ms = d["ms"] / d["launches"]
    bpl = d["bytes"] / d["launches"]
    fpl = d["flops"] / d["launches"]
    ipl = d["iops"] / d["launches"]
    t_hbm = bpl / (hbm_peak_gbs * 1e9)
    t_fp = fpl / FP64_PEAK_FLOPS
    t_int = ipl / INT_PEAK_OPS
    total = sum(v["ms"] for v in by.values())
    # The roofline of the path is HBM: a fused pass moves 32 B per amplitude.  The
    # arithmetic the kernel actually runs is reported beside it: FP64 flops against
    # the derived FP64 peak, or (Q60 engine) its wide integer multiply-adds against
    # the derived integer peak.
    ach = bpl / (per_ms * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": ach, "peak": hbm_peak_gbs, "unit": "GB/s", "frac": ach / hbm_peak_gbs}
    if ipl > 0:
        a_int = ipl / (per_ms * 1e-3) / 1e12
        out["alu"] = {"bound": "alu", "achieved": a_int, "peak": INT_PEAK_OPS / 1e12,
                      "unit": "T wide int multiply-adds/s", "frac": a_int / (INT_PEAK_OPS / 1e12),
                      "floor_ms_per_launch": t_int * 1e3}
    elif fpl > 0:
        a_fp = fpl / (per_ms * 1e-3) / 1e12
        out["alu"] = {"bound": "alu", "achieved": a_fp, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s (fp64)",
                      "frac": a_fp / (FP64_PEAK_FLOPS / 1e12), "floor_ms_per_launch": t_fp * 1e3}
    out.update({"kernel_kind": kind, "launches": d["launches"], "avg_launch_ms": per_ms,
                "share_of_kernel_time": d["ms"] / total if total else None,
                "algorithmic_bytes_per_launch": bpl, "algorithmic_flops_per_launch": fpl,
                "algorithmic_int_mads_per_launch": ipl,
                "hbm_floor_ms_per_launch": t_hbm * 1e3,
                "traffic": traffic_for(kind)})
    return out


def cpu_oracle_sample(n: int, gates: np.ndarray, budget_s: float = 20.0):
    """Oracle as it stands on the host cores: the first gates of the same circuit at
    the same n (the state is 2^n complex doubles), amp-updates/s."""
    import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    oracle.build()
    psi = oracle.zero_state(n)
    done = 0
    t0 = time.perf_counter()
    for k in range(len(gates)):
        oracle.apply_circuit(psi, n, gates[k:k + 1])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    del psi
    return {"value": done * float(1 << n) / dt, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "sample": f"first {done} of {len(gates)} gates at n={n} ({dt:.1f} s)", "seconds": dt}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    gates = w.layered_u3_cz(args.n, args.depth, 1)
    times, secs = [], []
    samp = None
    for i in range(args.warmup + args.steps):
        samp = cpu_oracle_sample(args.n, gates, budget_s=15.0 if i >= args.warmup else 3.0)
        if i >= args.warmup:
            times.append(samp["value"])
            secs.append(samp["seconds"])
    v = statistics.median(times)
    # a step of this arm is one bounded sample of the workload (the first gates of
    # the circuit); the whole circuit at the same rate is reported beside it
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(secs) * 1e3,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"layered U3+CZ brickwork, n={args.n}, depth {args.depth}", "n": args.n,
                       "full_circuit_ms_at_this_rate": len(gates) * float(1 << args.n) / v * 1e3},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": samp["cores"], "kind": "oracle",
                             "sample": samp["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batched_vqe(q, torch, steps: int, warmup: int, sets: int = 1024):
    """1024 parameter sets, n uniform in 10..20 (seed 3), 8-layer RY/RZ + CNOT-ring
    ansatz, TFIM h=0.7, angles uniform (seed 33): energy + adjoint gradient of every
    set per step, one persistent launch replayed from a CUDA graph.  (`sets` < 1024
    takes a smaller batch of the same recipe, for profiling.)"""
    ns = w.batch_qubit_counts(sets, 3)
    gl, npl, tl = [], [], []
    for n in ns:
        g, npar = w.hea_ansatz(int(n), 8)
        gl.append(g)
        npl.append(npar)
        tl.append(w.tfim(int(n), 0.7))
    params = w.uniform_angles(int(sum(npl)), 33)
    b = q.qs_batch_create(ns, gl, npl, tl)
    try:
        e = np.empty(len(ns))
        g = np.empty(len(params))
        for _ in range(warmup):
            q.qs_batch_run(b, params, e, g)
        t0 = time.perf_counter()
        kms = []
        for _ in range(steps):
            q.qs_batch_run(b, params, e, g)
            kms.append(q.qs_batch_last_ms(b))
        wall = (time.perf_counter() - t0) / steps
        info = q.qs_batch_info(b)
    finally:
        q.qs_batch_free(b)
    kms = float(np.mean(kms))
    # algorithmic traffic per step: per set (24 n forward gates + about 48 n backward
    # gate steps on two vectors + n + 1 for the Hamiltonian) sweeps of 32 B per amplitude
    sweep_bytes = float(sum((73 * int(n) + 1) * 32.0 * float(1 << int(n)) for n in ns))
    l2 = l2_copy_gbs(torch)
    eff = sweep_bytes / (kms * 1e-3) / 1e9
    return {"grad_evals_per_s": len(ns) / (kms * 1e-3), "kernel_ms": kms,
            "roofline": {"bound": "l2", "achieved": eff, "peak": l2, "unit": "GB/s", "frac": eff / l2,
                         "algorithmic_bytes_per_step": sweep_bytes,
                         "note": "logical gate-by-gate sweeps (per set: 73 n + 1 sweeps of 32 B per amplitude), "
                                 "on states that stay in L2 / shared memory (n <= 20: 16 MiB), against the "
                                 "copy bandwidth of a 2 x 24 MiB buffer pair measured in this run"},
            "e2e_grad_evals_per_s": len(ns) / wall, "e2e_ms": wall * 1e3, "sets": len(ns),
            "params": int(len(params)), "launch": info,
            "workload": f"{sets} sets, n~U{{10..20}}, 8-layer RY/RZ+CNOT-ring ansatz, TFIM h=0.7"}


def bench_adjoint(q, torch, stream, steps: int, hbm_peak: float):
    """Energy + 672-parameter adjoint gradient at n=28 (12-layer ansatz, ZZ chain).
    Roofline of the fused backward passes (the dominant kernel): each moves psi and
    lambda once, 64 B per amplitude (16 B read + 16 B written per vector)."""
    n = 28
    g, npar = w.hea_ansatz(n, 12)
    th = w.uniform_angles(npar, 4)
    H = w.zz_chain(n)
    h = q.qs_alloc(n, stream)
    try:
        q.qs_adjoint_grad(h, g, th, H)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            q.qs_adjoint_grad(h, g, th, H)
        dt = (time.perf_counter() - t0) / steps
        q.qs_timing_enable(h, True)
        q.qs_timing_fetch(h)
        q.qs_adjoint_grad(h, g, th, H)
        recs = q.qs_timing_fetch(h)
        q.qs_timing_enable(h, False)
    finally:
        q.qs_free(h)
    out = {"grad_evals_per_s": 1.0 / dt, "ms_per_eval": dt * 1e3, "n": n, "params": npar, "gates": len(g)}
    back = [r for r in recs if r["kind"] == 30 and r["k"] >= 2]
    fwd = [r for r in recs if r["kind"] == 11]
    total = sum(r["ms"] for r in recs)
    if back:
        bms = float(np.mean([r["ms"] for r in back]))
        gbs = 64.0 * float(1 << n) / (bms * 1e-3) / 1e9
        out["backward_pass"] = {"launches": len(back), "avg_ms": bms, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                                "share_of_kernel_time": sum(r["ms"] for r in back) / total,
                                "algorithmic_bytes_per_launch": 64.0 * float(1 << n)}
    if fwd:
        fms = float(np.mean([r["ms"] for r in fwd]))
        gbs = 32.0 * float(1 << n) / (fms * 1e-3) / 1e9
        out["forward_pass"] = {"launches": len(fwd), "avg_ms": fms, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak}
    return out


def l2_copy_gbs(torch, mib: int = 24, reps: int = 400) -> float:
    """Copy bandwidth of a buffer pair that fits in L2 (2 x 24 MiB of the 129 MB):
    read + written bytes / time, CUDA events, after warm-up."""
    a = torch.empty(mib << 18, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1.0)
    for _ in range(20):
        b.copy_(a)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.copy_(a)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return 2.0 * a.numel() * 4 / (ms * 1e-3) / 1e9


def bench_measure(q, torch, stream, hbm_peak: float):
    """Mid-circuit measurement at n=30 (16 GiB): the one-qubit marginal pass and
    the collapse pass of qs_measure, on the state after one U3 layer and the CZ
    brickwork, five qubits measured in turn.  Algorithmic bytes: marginal 16 B per
    amplitude read; collapse 8 B per amplitude read (the kept half) + 16 B written."""
    n = 30
    g = w.layered_u3_cz(n, 1, 1)
    h = q.qs_alloc(n, stream)
    try:
        q.qs_apply(h, g, None, None)
        q.qs_measure(h, 0, 0.5)
        q.qs_timing_enable(h, True)
        q.qs_timing_fetch(h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qubits = (29, 3, 17, 11, 24)
        for k, qb in enumerate(qubits):
            q.qs_measure(h, qb, 0.2 * k + 0.1)
        dt = (time.perf_counter() - t0) / len(qubits)
        recs = q.qs_timing_fetch(h)
        q.qs_timing_enable(h, False)
    finally:
        q.qs_free(h)
    N = float(1 << n)
    from paper_2212_14201_gb300 import _lib
    red = [r["ms"] for r in recs if r["kind"] == _lib.K_REDUCE]
    col = [r["ms"] for r in recs if r["kind"] == _lib.K_OTHER]
    out = {"n": n, "ms_per_measurement": dt * 1e3, "measurements_per_s": 1.0 / dt}
    if red:
        ms = float(np.mean(red))
        out["marginal"] = {"avg_ms": ms, "gbs": 16 * N / (ms * 1e-3) / 1e9, "frac_of_hbm": 16 * N / (ms * 1e-3) / 1e9 / hbm_peak}
    if col:
        ms = float(np.mean(col))
        out["collapse"] = {"avg_ms": ms, "gbs": 24 * N / (ms * 1e-3) / 1e9, "frac_of_hbm": 24 * N / (ms * 1e-3) / 1e9 / hbm_peak}
    return out


def bench_reductions(q, torch, stream, hbm_peak: float, reps: int = 3, n: int = 30):
    """Rows A6-A8 on the output state of the config-1 circuit (n=30: 16 GiB):
    squared norm, one-qubit marginal, <Z_i> for all n qubits, a TFIM Pauli sum
    ((n-1) ZZ + n X terms, h = 0.7) and 10^6 samples, each timed with CUDA events
    on the state's stream.  Bytes: 16 B per amplitude read for the norm, marginal
    and <Z_i>; for the Pauli sum 16 B per amplitude per pass of the tile kernel,
    which reads the state once per pass (the passes are counted from the
    library's kernel log; n=30: 5, tiles spanning 12, 8, 8 and 2 of the X masks)."""
    g = w.layered_u3_cz(n, 20, 1)
    terms = w.tfim(n, 0.7)
    h = q.qs_alloc(n, stream)
    N = float(1 << n)
    out = {"n": n}
    try:
        p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
        q.qs_apply(h, g, None, p)
        q.qs_plan_free(p)
        q.qs_timing_enable(h, True)
        q.qs_expect_pauli(h, terms)
        pauli_passes = sum(1 for r in q.qs_timing_fetch(h) if r["kind"] == q._lib.K_REDUCE)
        q.qs_timing_enable(h, False)
        out["pauli_passes"] = pauli_passes
        dev = torch.empty(64, dtype=torch.float64, device="cuda")
        samples = torch.empty(1_000_000, dtype=torch.int64, device="cuda")

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        cases = {
            "norm": (lambda: q.qs_probs(h, [], dev), 16 * N),
            "marginal_1q": (lambda: q.qs_probs(h, [17], dev), 16 * N),
            "expect_z_all": (lambda: q.qs_expect_z_all(h), 16 * N),
            "expect_pauli_tfim": (lambda: q.qs_expect_pauli(h, terms), 16 * N * pauli_passes),
            "sample_1e6": (lambda: q.qs_sample(h, 11, 1_000_000, samples), 16 * N),
        }
        for name, (fn, nbytes) in cases.items():
            ms = timed(fn)
            gbs = nbytes / (ms * 1e-3) / 1e9
            out[name] = {"ms": ms, "gbs": gbs, "frac_of_hbm": gbs / hbm_peak}
    finally:
        q.qs_free(h)
    return out


# FP32 peak derived from unit counts and clock: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz.
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2.07e9


def bench_c64(q, torch, stream, hbm_peak: float, steps: int = 3):
    """The complex64 variant on the config-1 circuit (n=30, 8 GiB state): greedy
    plan, FP32 tile passes.  Algorithmic bytes per tile pass: 16 per amplitude
    (8 read + 8 written); flops per amplitude: 14 per U3."""
    from paper_2212_14201_gb300 import _lib
    n = 30
    g = w.layered_u3_cz(n, 20, 1)
    p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
    h = q.qs_alloc_c64(n, stream)
    try:
        q.qs_apply(h, g, None, p)
        q.qs_timing_enable(h, True)
        q.qs_timing_fetch(h)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            q.qs_set_zero(h)
            q.qs_apply(h, g, None, p)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        recs = q.qs_timing_fetch(h)
        q.qs_timing_enable(h, False)
        norm2 = float(q.qs_probs(h, [])[0])
    finally:
        q.qs_free(h)
        q.qs_plan_free(p)
    tiles = [r for r in recs if r["kind"] == _lib.K_TILE]
    out = {"n": n, "gates": len(g), "ms_per_apply": ms, "amp_updates_per_s": len(g) * float(1 << n) / (ms * 1e-3),
           "norm2": norm2}
    if tiles:
        tms = float(np.mean([r["ms"] for r in tiles]))
        fl = float(np.mean([r["flops"] for r in tiles]))
        gbs = 16.0 * float(1 << n) / (tms * 1e-3) / 1e9
        tf = fl / (tms * 1e-3) / 1e12
        out["tile_pass"] = {"avg_ms": tms, "launches_per_apply": len(tiles) // steps,
                            "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                            "fp32_tflops": tf, "fp32_frac": tf / (FP32_PEAK_FLOPS / 1e12)}
    return out


def bench_noisy(q, torch, stream):
    """Noise trajectories on the n=28 brickwork (depth 20, 830 gates): depolarizing
    p=1e-3 on every gate (scaled-unitary channel: Paulis join the fused gate
    stream), then the same plus amplitude damping p=1e-3 on every CZ (one weight
    reduction and one renormalised Kraus pass per touched qubit)."""
    n = 28
    g = w.layered_u3_cz(n, 20, 1)
    out = {"n": n, "gates": len(g)}
    cases = {"depolarizing": w.noise_rules([w.noise_rule("DEPOLARIZING", None, 1e-3)]),
             "depolarizing+damping": w.noise_rules([w.noise_rule("DEPOLARIZING", None, 1e-3),
                                                    w.noise_rule("DAMPING", "CZ", 1e-3)])}
    h = q.qs_alloc(n, stream)
    try:
        for name, rules in cases.items():
            q.qs_run_noisy(h, g, rules, seed=0)
            ts = []
            for seed in (1, 2):
                q.qs_set_zero(h)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                nd = q.qs_run_noisy(h, g, rules, seed=seed)
                ts.append(time.perf_counter() - t0)
            out[name] = {"ms_per_trajectory": 1e3 * float(np.mean(ts)), "draws": nd}
        p = q.qs_plan_create(n, g, q.PLAN_GREEDY, 5)
        q.qs_set_zero(h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.qs_apply(h, g, None, p)
        torch.cuda.synchronize()
        out["noiseless_fused_ms"] = 1e3 * (time.perf_counter() - t0)
        q.qs_plan_free(p)
    finally:
        q.qs_free(h)
    return out


def bench_partial(q, torch):
    """Partial amplitudes at n=40 (a 16 TiB state): the depth-20 brickwork cut
    between qubits 19 and 20 (10 CZ cuts, 1024 paths of two 20-qubit blocks),
    10^6 random basis indices (seed 5)."""
    n = 40
    g = w.layered_u3_cz(n, 20, 1)
    idx = np.random.Generator(np.random.PCG64(5)).integers(0, 1 << n, 1_000_000, dtype=np.uint64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    amps, paths = q.qs_partial_amplitudes(n, g, 20, idx)
    dt = time.perf_counter() - t0
    return {"n": n, "gates": len(g), "paths": paths, "amplitudes": len(idx), "s": dt,
            "amplitudes_per_s": len(idx) / dt, "mean_p_times_2n": float(np.mean(np.abs(amps) ** 2)) * 2.0 ** n}


def bench_learned_plan(q, torch, stream):
    """n=32 (64 GiB), 2000 random gates (40 % two-qubit, seed 2): greedy plan vs
    the learned plan (cost model from paper_2212_14201_gb300/costmodel_weights.json)
    vs plain per-gate apply, one timed apply each after one untimed."""
    from paper_2212_14201_gb300 import costmodel
    n = 32
    g = w.random_circuit(n, 2000, 2, two_qubit_prob=0.4)
    model = costmodel.load()
    if model is None:
        return {"skipped": "no trained cost model weights"}
    out = {"n": n, "gates": len(g)}
    h = q.qs_alloc(n, stream)
    try:
        plans = {"greedy": q.qs_plan_create(n, g, q.PLAN_GREEDY, 5), "learned": q.qs_plan_create_learned(n, g, model),
                 "plain": None}
        for name, p in plans.items():
            q.qs_set_zero(h)
            q.qs_apply(h, g, None, p)
            q.qs_set_zero(h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            q.qs_apply(h, g, None, p)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st = q.qs_plan_get_stats(p) if p else {}
            out[name] = {"ms": ms, "amp_updates_per_s": len(g) * float(1 << n) / (ms * 1e-3),
                         "passes": st.get("n_passes"), "tile_qubits": st.get("tile_qubits")}
        out["norm2"] = float(q.qs_probs(h, [])[0])
        out["learned_gain_vs_greedy"] = out["greedy"]["ms"] / out["learned"]["ms"]
        out["learned_gain_vs_plain"] = out["plain"]["ms"] / out["learned"]["ms"]
        for p in plans.values():
            if p:
                q.qs_plan_free(p)
    finally:
        q.qs_free(h)
    # a held-out n=30 random circuit (600 gates, 40 % two-qubit, seed 302): best of two applies per plan
    try:
        n2 = 30
        g2 = w.random_circuit(n2, 600, 302, two_qubit_prob=0.4)
        h2 = q.qs_alloc(n2, stream)
        held = {"n": n2, "gates": len(g2), "seed": 302}
        try:
            for name, p in (("greedy", q.qs_plan_create(n2, g2, q.PLAN_GREEDY, 5)),
                            ("learned", q.qs_plan_create_learned(n2, g2, model))):
                best = 1e30
                for _ in range(3):
                    q.qs_set_zero(h2)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    q.qs_apply(h2, g2, None, p)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                held[name] = {"ms": best, "passes": q.qs_plan_get_stats(p)["n_passes"]}
                q.qs_plan_free(p)
            held["learned_gain_vs_greedy"] = held["greedy"]["ms"] / held["learned"]["ms"]
        finally:
            q.qs_free(h2)
        out["held_out_n30"] = held
    finally:
        q.qs_mlp_free(model)
    return out


def run_ours(args, world, rank, local, pg):
    import torch

    import paper_2212_14201_gb300 as q
    q.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    if args.only_batch:
        if rank == 0:
            print(json.dumps({"batched_vqe": bench_batched_vqe(q, torch, args.steps, args.warmup, args.batch_sets)}))
        return
    if args.only_reductions:
        if rank == 0:
            print(json.dumps({"reductions": bench_reductions(q, torch, stream, peaks()[0], n=args.only_reductions)}))
        return
    n = args.n
    gates = w.layered_u3_cz(n, args.depth, 1)
    ng = len(gates)
    hbm_peak, peak_src = peaks()

    h = q.qs_alloc(n, stream)
    norm_out = torch.empty(1, dtype=torch.float64, device="cuda")
    samples = torch.empty(SHOTS, dtype=torch.int64, device="cuda")
    plan = None
    plan_stats = None
    plan_ms = None
    try:
        t_plan = time.perf_counter()
        plan = q.qs_plan_create(n, gates, q.PLAN_GREEDY, 5)
        plan_ms = (time.perf_counter() - t_plan) * 1e3
        plan_stats = q.qs_plan_get_stats(plan)
    except q.QsimError:
        plan = None

    def step(p):
        q.qs_set_zero(h)
        q.qs_apply(h, gates, None, p)
        q.qs_probs(h, [], norm_out)
        q.qs_sample(h, SAMPLE_SEED, SHOTS, samples)

    def timed(p, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            step(p)
        torch.cuda.synchronize()
        barrier(pg)
        torch.cuda.synchronize()
        q.qs_timing_enable(h, True)
        q.qs_timing_fetch(h)
        l0 = q.qs_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(local)
        if sample_clocks:
            clk.__enter__()
        e0.record(stream)
        for _ in range(steps):
            step(p)
        e1.record(stream)
        torch.cuda.synchronize()
        if sample_clocks:
            clk.__exit__()
        barrier(pg)
        torch.cuda.synchronize()
        launches = q.qs_launch_count() - l0
        recs = q.qs_timing_fetch(h)
        q.qs_timing_enable(h, False)
        ms = e0.elapsed_time(e1) / steps
        return max_over_ranks(pg, ms), recs, launches, (clk.summary() if sample_clocks else None)

    ms, recs, launches, clocks = timed(plan, args.steps, args.warmup, sample_clocks=True)
    norm2 = float(norm_out.item())
    fused_samples = samples.cpu().numpy().astype(np.uint64)  # the plain runs below reuse `samples`
    amp_updates = ng * float(1 << n)
    value = whole_job_value(world, amp_updates, ms)
    roof = roofline(recs, hbm_peak)
    gate_bytes = sum(r["items"] * 32.0 for r in recs if r["kind"] in (1, 2, 3, 4, 5, 10, 11))
    step_gate_ms = sum(r["ms"] for r in recs if r["kind"] in (1, 2, 3, 4, 5, 10, 11)) / args.steps

    plain = None
    plain_fp64 = None
    if plan is not None and not args.no_plain:
        ksteps = max(1, args.steps - 1)
        pms, precs, _, _ = timed(None, ksteps, 1)
        pb = sum(r["items"] * 32.0 for r in precs if r["kind"] in (1, 2, 3, 4, 5))
        pg_ms = sum(r["ms"] for r in precs if r["kind"] in (1, 2, 3, 4, 5)) / ksteps
        plain = {"value": whole_job_value(world, amp_updates, pms), "ms_per_step": pms,
                 "hbm_gbs_algorithmic": pb / ksteps / (pg_ms * 1e-3) / 1e9,
                 "roofline": roofline(precs, hbm_peak)}
        # the same per-gate kernels with IEEE FP64 arithmetic (context: the FP64 pipe bound)
        q.qs_set_arith(h, q.ARITH_FP64)
        fms, frecs, _, _ = timed(None, 1, 1)
        q.qs_set_arith(h, q.ARITH_AUTO)
        plain_fp64 = {"value": whole_job_value(world, amp_updates, fms), "ms_per_step": fms,
                      "roofline": roofline(frecs, hbm_peak)}

    # end to end through the public API: host gate list in, norm and samples out to host
    host_samples = np.empty(SHOTS, dtype=np.uint64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q.qs_set_zero(h)
        q.qs_apply(h, gates, None, plan)
        nn = q.qs_probs(h, [])
        q.qs_sample(h, SAMPLE_SEED, SHOTS, host_samples)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(pg, e2e_s)
    ok_e2e = np.array_equal(host_samples, fused_samples) and abs(nn[0] - norm2) == 0.0

    if plan is not None:
        q.qs_plan_free(plan)
    q.qs_free(h)

    extra = {}
    if not args.no_extra:
        torch.cuda.empty_cache()
        extra["batched_vqe"] = bench_batched_vqe(q, torch, 3, 3)
        extra["adjoint_n28"] = bench_adjoint(q, torch, stream, 2, hbm_peak)
        extra["measure_n30"] = bench_measure(q, torch, stream, hbm_peak)
        extra["reductions_n30"] = bench_reductions(q, torch, stream, hbm_peak)
        extra["c64_n30"] = bench_c64(q, torch, stream, hbm_peak)
        extra["noisy_n28"] = bench_noisy(q, torch, stream)
        extra["partial_n40"] = bench_partial(q, torch)
        if not args.no_n32:
            try:
                extra["learned_n32"] = bench_learned_plan(q, torch, stream)
            except q.QsimError as ex:
                extra["learned_n32"] = {"skipped": str(ex)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = cpu_oracle_sample(n, gates)
        except Exception as ex:  # host RAM too small for the state, for example
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"not run: {ex}"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64",
        "dtype_note": "complex128 state in HBM; gate arithmetic in Q60 fixed point (int64 limbs, 2^-60 "
                      "resolution) on the integer pipe; the squared norm as exact integer sums of the Q60 "
                      "squares; sampling in f64 by its canonical definition",
        "data": "synthetic",
        "config": {"workload": f"layered U3+CZ brickwork, n={n}, depth {args.depth} ({ng} gates), "
                               f"norm + {SHOTS} samples", "n": n, "gates": ng, "shots": SHOTS,
                   "mode": "fused" if plan is not None else "plain", "plan": plan_stats,
                   "l2": "state (16 GiB at n=30) is larger than L2", "parallelism": f"replicas x{world}"},
        "hbm_gbs": gate_bytes / (step_gate_ms * 1e-3) / 1e9 if step_gate_ms else None,
        "hbm_gbs_note": "algorithmic bytes of the gate kernels / their device time",
        "norm2": norm2,
        "plain": plain,
        "plain_fp64": plain_fp64,
        "roofline": roof,
        "peak_source": {"hbm": peak_src, "fp64": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"},
        "cpu_baseline": cpu,
        "e2e": {"value": world * amp_updates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(gates.nbytes),
                "d2h_bytes_per_step": SHOTS * 8 + 8, "matches_device_run": bool(ok_e2e),
                "plan_ms": plan_ms,
                "plan_note": "the greedy plan is built once before the timed steps (host, plan_ms) and reused; "
                             "each step's op lists and phase tables are rebuilt on the host from the gate list"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "batched_vqe": extra.get("batched_vqe"),
        "adjoint_n28": extra.get("adjoint_n28"),
        "learned_n32": extra.get("learned_n32"),
        "measure_n30": extra.get("measure_n30"),
        "reductions_n30": extra.get("reductions_n30"),
        "c64_n30": extra.get("c64_n30"),
        "noisy_n28": extra.get("noisy_n28"),
        "partial_n40": extra.get("partial_n40"),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
