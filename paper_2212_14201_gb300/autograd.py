"""torch.autograd binding of the adjoint-gradient kernel.

`expectation(params, gates, terms, n)` returns E(params) = <psi(params)|H|psi(params)>
as a 0-d float64 tensor that carries a gradient: the forward call runs
qs_adjoint_grad (the forward sweep, H psi and the fused backward sweep) and keeps
dE/dparams for backward, which scales it by the incoming gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


class _Expectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, gates, terms, handle):
        p = params.detach().to("cpu", torch.float64).contiguous().numpy()
        energy, grad = _lib.qs_adjoint_grad(handle, gates, p, terms)
        ctx.save_for_backward(torch.from_numpy(grad).to(params.device, params.dtype))
        return torch.tensor(energy, dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None


class Expectation:
    """Callable E(params) for a fixed circuit and Hamiltonian on an n-qubit state
    owned by the library (re-used across calls)."""

    def __init__(self, n: int, gates, terms, stream=None):
        self.n = n
        self.gates = _lib.as_gates(gates)
        self.terms = _lib.as_paulis(terms)
        self.handle = _lib.qs_alloc(n, stream if stream is not None else torch.cuda.current_stream())

    def __call__(self, params: torch.Tensor) -> torch.Tensor:
        return _Expectation.apply(params, self.gates, self.terms, self.handle)

    def close(self):
        if self.handle:
            _lib.qs_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expectation(params: torch.Tensor, gates, terms, n: int) -> torch.Tensor:
    e = Expectation(n, gates, terms)
    try:
        return e(params)
    finally:
        e.close()


__all__ = ["Expectation", "expectation", "np"]
