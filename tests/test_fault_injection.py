"""Host-side fault injection (qs_fault_set, QS_FAULT): the library's allocation
and launch error paths, driven without any GPU fault.

CPU tests: the hook's arming rules, the QS_FAULT environment parser, and the
allocation leg of the entry points that allocate before touching the device
(qs_alloc, qs_alloc_external).  GPU tests: qs_mlp_create, and every entry point
that takes a state, under an allocation fault and under a launch fault -- the
call reports QS_ERR_OOM / QS_ERR_CUDA, a call that only reads the state leaves
it bit-identical, and every state is usable again once the fault is disarmed."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OOM, CUDA, INVALID = -2, -3, -1
TAG = "(injected by the armed fault)"


@pytest.fixture(scope="module")
def lib():
    import paper_2212_14201_gb300 as q
    q.build()
    yield q
    q.qs_fault_set(q.FAULT_NONE)


@pytest.fixture(autouse=True)
def disarm(lib):
    lib.qs_fault_set(lib.FAULT_NONE)
    yield
    lib.qs_fault_set(lib.FAULT_NONE)


def test_arming_rules(lib):
    q = lib
    for bad in ((7, 0, 1), (q.FAULT_ALLOC, -1, 1), (q.FAULT_ALLOC, 0, 0), (q.FAULT_LAUNCH, 0, -2)):
        with pytest.raises(q.QsimError) as ei:
            q.qs_fault_set(*bad)
        assert ei.value.code == INVALID
    q.qs_fault_set(q.FAULT_LAUNCH, 3, 2)
    assert q.qs_fault_get() == {"kind": q.FAULT_LAUNCH, "after": 3, "left": 2, "fired": 0, "env_status": 0}
    q.qs_fault_set(q.FAULT_NONE)
    assert q.qs_fault_get()["kind"] == q.FAULT_NONE


def test_alloc_fault_fails_state_creation(lib):
    q = lib
    q.qs_fault_set(q.FAULT_ALLOC, 0, 2)
    for _ in range(2):
        with pytest.raises(q.QsimError) as ei:
            q.qs_alloc(10)
        assert ei.value.code == OOM and TAG in str(ei.value)
    st = q.qs_fault_get()
    assert st["fired"] == 2 and st["left"] == 0
    # the fault is spent: the next creation reaches CUDA (no device here: a CUDA
    # error; on a GPU machine: a state), never an injected failure
    try:
        h = q.qs_alloc(10)
    except q.QsimError as e:
        assert TAG not in str(e)
    else:
        q.qs_free(h)
    assert q.qs_fault_get()["fired"] == 2


def test_alloc_fault_skips_events_before_after(lib):
    """after=1: qs_alloc_external allocates only the workspace, so with an external
    buffer the first allocation passes to CUDA and only a later one is injected;
    handles are never returned on failure."""
    q = lib
    lib_ = q._lib.lib()
    q.qs_fault_set(q.FAULT_ALLOC, 0, 1)
    out = ctypes.c_void_p(12345)
    # an external buffer is only stored, never dereferenced, before the workspace
    # allocation fails
    rc = lib_.qs_alloc_external(8, ctypes.c_void_p(1 << 20), None, ctypes.byref(out))
    assert rc == OOM and out.value is None
    assert TAG in q.qs_last_error()
    q.qs_fault_set(q.FAULT_ALLOC, 1, 1)
    out = ctypes.c_void_p(12345)
    rc = lib_.qs_alloc(8, None, ctypes.byref(out))
    # first event (the state buffer) went to CUDA: either it failed there (no
    # device) or the second (workspace) was injected
    st = q.qs_fault_get()
    if rc == OOM and TAG in q.qs_last_error():
        assert st["fired"] == 1 and out.value is None
    else:
        assert st["fired"] == 0
        if rc == 0:
            lib_.qs_free(out)


@pytest.mark.gpu
def test_alloc_fault_in_model_creation(lib):
    """qs_mlp_create creates its stream before allocating, so this leg needs a GPU."""
    q = lib
    q.qs_fault_set(q.FAULT_ALLOC, 0, -1)
    with pytest.raises(q.QsimError) as ei:
        q.qs_mlp_create(4, 8, None, 1)
    assert ei.value.code == OOM and TAG in str(ei.value)
    assert q.qs_fault_get()["left"] == -1


@pytest.mark.parametrize("spec,want", [
    ("alloc", (1, 0, 1, 0)),
    ("launch:5", (2, 5, 1, 0)),
    ("alloc:2:-1", (1, 2, -1, 0)),
    ("launch:0:3", (2, 0, 3, 0)),
    ("bogus", (0, 0, 0, INVALID)),
    ("alloc:-1", (0, 0, 0, INVALID)),
])
def test_environment_spec(lib, spec, want):
    """QS_FAULT arms the fault when the library loads (a fresh process)."""
    code = ("import paper_2212_14201_gb300 as q, json; s = q.qs_fault_get(); "
            "print(json.dumps([s['kind'], s['after'], s['left'], s['env_status']]))")
    env = dict(os.environ, QS_FAULT=spec)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    import json
    assert tuple(json.loads(r.stdout.strip().splitlines()[-1])) == want


# ---- GPU: every entry point that takes a state -------------------------------------

N_GPU = 12


def _read_calls(q, w):
    """Calls that only read the state: (name, call(h) -> comparable result)."""
    H = w.tfim(N_GPU)
    sub = [0, 3, 7]
    return [
        ("probs", lambda h: q.qs_probs(h, sub)),
        ("probs_full", lambda h: q.qs_probs(h, list(range(N_GPU)))),
        ("probs_dict", lambda h: sorted(q.qs_probs_dict(h, sub, 1e-3).items())),
        ("expect_z_all", lambda h: q.qs_expect_z_all(h)),
        ("expect_pauli", lambda h: q.qs_expect_pauli(h, H)),
        ("sample_host", lambda h: q.qs_sample(h, 5, 4096)),
        ("get_state", lambda h: q.qs_get_state(h)),
    ]


def _write_calls(q, w):
    """Calls that write the state: (name, call(h))."""
    g = w.random_circuit(N_GPU, 120, 11, two_qubit_prob=0.4)
    hea, npar = w.hea_ansatz(N_GPU, 2)
    th = w.uniform_angles(npar, 3)
    prog, pg = w.random_program(N_GPU, 4)
    rules = w.noise_rules([w.noise_rule("DEPOLARIZING", None, 0.05)])

    def greedy(h):
        p = q.qs_plan_create(N_GPU, g, q.PLAN_GREEDY, 5)
        try:
            q.qs_apply(h, g, None, p)
        finally:
            q.qs_plan_free(p)
    return [
        ("apply_plain", lambda h: q.qs_apply(h, g)),
        ("apply_greedy", greedy),
        ("set_zero", lambda h: q.qs_set_zero(h)),
        ("measure", lambda h: q.qs_measure(h, 2, 0.4)),
        ("adjoint_grad", lambda h: q.qs_adjoint_grad(h, hea, th, w.zz_chain(N_GPU))),
        ("run_program", lambda h: q.qs_run_program(h, prog, pg, seed=2)),
        ("run_noisy", lambda h: q.qs_run_noisy(h, g, rules, seed=4)),
    ]


def _same(a, b):
    if isinstance(a, tuple):
        return all(_same(x, y) for x, y in zip(a, b))
    if isinstance(a, list):
        return a == b
    return np.array_equal(np.asarray(a), np.asarray(b))


@pytest.fixture(scope="module")
def gpu_state(lib):
    import torch
    assert torch.cuda.is_available()
    import workloads as w
    q = lib
    h = q.qs_alloc(N_GPU, torch.cuda.current_stream())
    g = w.random_circuit(N_GPU, 200, 21, two_qubit_prob=0.4)
    q.qs_apply(h, g)
    ref = q.qs_get_state(h)
    yield q, w, h, g, ref
    q.qs_free(h)


def _restore(q, h, g, ref):
    q.qs_fault_set(q.FAULT_NONE)
    q.qs_set_zero(h)
    q.qs_apply(h, g)
    assert np.array_equal(q.qs_get_state(h), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["alloc", "launch"])
def test_read_calls_leave_state_unchanged(gpu_state, kind):
    q, w, h, g, ref = gpu_state
    fk = q.FAULT_ALLOC if kind == "alloc" else q.FAULT_LAUNCH
    code = OOM if kind == "alloc" else CUDA
    fired_any = False
    for name, call in _read_calls(q, w):
        _restore(q, h, g, ref)
        want = call(h)
        q.qs_fault_set(fk, 0, -1)
        try:
            call(h)
        except q.QsimError as e:
            assert e.code == code and TAG in str(e), (name, str(e))
            fired_any = True
        else:
            assert q.qs_fault_get()["fired"] == 0, name   # succeeded only if nothing fired
        q.qs_fault_set(q.FAULT_NONE)
        assert np.array_equal(q.qs_get_state(h), ref), name
        assert _same(call(h), want), name
    assert fired_any


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["alloc", "launch"])
def test_write_calls_report_and_recover(gpu_state, kind):
    q, w, h, g, ref = gpu_state
    fk = q.FAULT_ALLOC if kind == "alloc" else q.FAULT_LAUNCH
    code = OOM if kind == "alloc" else CUDA
    for name, call in _write_calls(q, w):
        _restore(q, h, g, ref)
        q.qs_fault_set(fk, 0, -1)
        try:
            call(h)
        except q.QsimError as e:
            assert e.code == code and TAG in str(e), (name, str(e))
        else:
            assert q.qs_fault_get()["fired"] == 0, name
        # the handle stays valid: it is reset and reproduces the reference state
        _restore(q, h, g, ref)
        if kind == "launch":
            # every one of these calls launches a kernel, so a launch fault always fires
            q.qs_fault_set(fk, 0, 1)
            with pytest.raises(q.QsimError):
                call(h)
            _restore(q, h, g, ref)


@pytest.mark.gpu
def test_later_launch_fault_mid_call(gpu_state):
    """The third launch check of a multi-kernel apply fails: the call reports it,
    the kernels already queued complete, and the state recovers."""
    q, w, h, g, ref = gpu_state
    _restore(q, h, g, ref)
    q.qs_fault_set(q.FAULT_LAUNCH, 2, 1)
    with pytest.raises(q.QsimError) as ei:
        q.qs_apply(h, g)
    assert ei.value.code == CUDA and q.qs_fault_get()["fired"] == 1
    q.qs_sync(h)
    _restore(q, h, g, ref)
