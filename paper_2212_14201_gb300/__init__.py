"""GB300-native full-amplitude state-vector simulator (QPanda's full-amplitude
virtual machine, arXiv 2212.14201) behind the C ABI in include/qsim.h.

`paper_2212_14201_gb300._lib` has one wrapper per C entry point (same names).
`StateVector` is a convenience handle whose amplitudes live in a PyTorch CUDA
tensor (torch provides device memory and the stream; all arithmetic runs in the
library's kernels).
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (qs_plan_create_tiled, qs_batch_create, qs_batch_free, qs_batch_info, qs_batch_last_ms, qs_batch_run,  # noqa: F401
                   ARITH_AUTO, ARITH_FIXED, ARITH_FP64, qs_adjoint_grad, qs_set_arith,
                   qs_state_modified,
                   GATE_DTYPE, PAULI_DTYPE, PLAN_GREEDY, PLAN_LEARNED, PLAN_PLAIN, QsimError,  # noqa: F401
                   qs_alloc, qs_alloc_external, qs_apply, qs_apply_matrix, qs_device_ptr, qs_expect_pauli,
                   qs_expect_z_all, qs_free, qs_gate_list_dagger, qs_get_state, qs_last_error, qs_max_qubits,
                   qs_num_qubits, qs_plan_create, qs_plan_free, qs_plan_get_stats, qs_probs, qs_probs_dict,
                   qs_plan_pass_info, qs_plan_passes, qs_sample, qs_set_state, qs_set_zero, qs_sync, qs_timing_enable, qs_timing_fetch,
                   qs_launch_count)


def build(verbose: bool = False, force: bool = False) -> str:
    from .buildlib import build as _b
    return _b(verbose=verbose, force=force)


class StateVector:
    """n-qubit complex128 state in a torch CUDA tensor, |0...0> on creation."""

    def __init__(self, n: int, device=None, stream=None):
        import torch
        self.n = n
        dev = torch.device("cuda" if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        with torch.cuda.device(dev):
            self.amps = torch.empty(2 << n, dtype=torch.float64, device=dev)
        self.handle = qs_alloc_external(n, self.amps, self.stream)
        qs_set_zero(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            qs_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- thin forwards --------------------------------------------------------------
    def apply(self, gates, params=None, plan=None):
        qs_apply(self.handle, gates, params, plan)
        return self

    def apply_matrix(self, targets, mat, ctrl_mask=0):
        qs_apply_matrix(self.handle, targets, mat, ctrl_mask)
        return self

    def set_state(self, amps):
        qs_set_state(self.handle, amps)

    def state(self) -> np.ndarray:
        return qs_get_state(self.handle)

    def probs(self, qubits=None, out=None):
        return qs_probs(self.handle, qubits, out)

    def probs_dict(self, qubits=None, threshold=0.0):
        return qs_probs_dict(self.handle, qubits, threshold)

    def expect_z(self):
        return qs_expect_z_all(self.handle)

    def expect(self, terms):
        return qs_expect_pauli(self.handle, terms)

    def sample(self, seed, shots, out=None):
        return qs_sample(self.handle, seed, shots, out)

    def sync(self):
        qs_sync(self.handle)
