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
from ._lib import (ARITH_AUTO, ARITH_FIXED, ARITH_FP64, FAULT_ALLOC, FAULT_LAUNCH, FAULT_NONE, GATE_DTYPE, NOISE_DTYPE, PAULI_DTYPE, PINSTR_DTYPE, PLAN_GREEDY,  # noqa: F401
                   PLAN_LEARNED, PLAN_PLAIN, QsimError)

# every C entry point's wrapper, under its C name
for _name in dir(_lib):
    if _name.startswith("qs_"):
        globals()[_name] = getattr(_lib, _name)
del _name


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
