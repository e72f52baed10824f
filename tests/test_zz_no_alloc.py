"""The allocation-free <Z_i> entry point (qs_expect_z_all_noalloc).

It serves callers that cannot call cudaMalloc, such as code whose device memory
belongs to another allocator or code on a latency-critical path.  Its scratch
is a file-scope device array instead of an allocation.  This test calls it
through the C ABI with caller-owned device buffers, twice in a row on different
states, and checks each result against the allocating entry point qs_expect_z_all.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu
TOL = 1e-12


def test_noalloc_expect_z_matches_allocating_entry_point_and_oracle():
    import torch
    assert torch.cuda.is_available()
    import paper_2212_14201_gb300 as q
    q.build()
    lib = q._lib.lib()
    stream = torch.cuda.current_stream()
    import oracle as orc
    orc.build()
    # a small n right after a larger one: fewer CTAs run over partials that the
    # larger call left in the shared array
    for n, seed in ((14, 1), (20, 2), (9, 3)):
        g = w.random_circuit(n, 150, seed, two_qubit_prob=0.4)
        h = q.qs_alloc(n, stream)
        try:
            q.qs_apply(h, g)
            want = q.qs_expect_z_all(h)
            amps = torch.empty(2 << n, dtype=torch.float64, device="cuda")
            q.qs_get_state(h, amps)
        finally:
            q.qs_free(h)
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.qs_expect_z_all_noalloc(ctypes.c_void_p(amps.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, q.qs_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert float(np.max(np.abs(got - want))) < TOL
        # the floating-point reduction it runs, against the CPU oracle on the same state
        st = amps.cpu().numpy()
        assert float(np.max(np.abs(got - orc.expect_z(st, n)))) < TOL


def test_noalloc_rejects_sizes_outside_its_range():
    import torch
    import paper_2212_14201_gb300 as q
    lib = q._lib.lib()
    buf = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lib.qs_expect_z_all_noalloc(ctypes.c_void_p(buf.data_ptr()), 35, ctypes.c_void_p(buf.data_ptr()), None)
    assert rc == -1 and "n <= 34" in q.qs_last_error()
