"""Element-wise gradient tolerance shared by the GPU gradient tests.

A gradient entry g_k = 2 Im<lambda_k|G_k|psi_k> (adjoint method) is compared
element by element: |a - b| <= 1e-9 |b| + floor.  The absolute floor covers the
entries whose exact value is zero or tiny (for example the last layer's RZ
parameters before a Z-diagonal observable: their gradient vanishes identically,
and any computed value is rounding noise).  The floor is derived from the
arithmetic, not fitted:

  e_op  2-norm error one applied op adds to a state of norm 1:
        FP64  each component is formed from at most four products and three
              additions, relative error <= 4u per component (u = 2^-53), so
              e_op <= 8u with a factor 2 to spare;
        Q60   each component carries at most 7 * 2^-60 absolute error (six
              dropped low-limb products and the rounding) plus the conversion,
              so e_op <= 8 * 2^-60 * sqrt(2^(n+1)) (the absolute error of every
              one of the 2^(n+1) real components).
  The oracle (FP64) and the GPU engine each contribute an e_op.  Rounding errors
  of different ops are independent and of mean (close to) zero, so after G ops
  the error vectors of psi and lambda have 2-norm ~ sqrt(G) e_op (lambda's scaled
  by ||H||_1, the sum of |coefficients|); their inner product with the other,
  fixed, unit vector picks up ~ 1/sqrt(2^n) of that norm.  Hence
      |dg_k| ~ 4 ||H||_1 sqrt(G) e_op / sqrt(2^n),
  and the floor is 100 times that estimate.  (The worst-case bound, with G for
  sqrt(G) and without the 1/sqrt(2^n), is far looser than any observed error.)
"""
from __future__ import annotations

import math

import numpy as np

U = 2.0 ** -53


def e_op(n: int) -> float:
    """Per-op 2-norm error of the GPU engine (the larger of FP64 and Q60) plus the oracle's."""
    return max(8.0 * U, 8.0 * 2.0 ** -60 * math.sqrt(2.0 ** (n + 1))) + 8.0 * U


def grad_floor(n: int, n_ops: int, h1: float) -> float:
    return 100.0 * 4.0 * max(h1, 1.0) * math.sqrt(max(n_ops, 1)) * e_op(n) / math.sqrt(2.0 ** n)


def h1_of(terms) -> float:
    """||H||_1 of a Pauli-term array (sum of |coefficients|)."""
    return float(np.sum(np.abs(np.asarray(terms["coef"], dtype=np.float64))))


def grad_close(a, b, n: int, n_ops: int, h1: float, rel: float = 1e-9) -> bool:
    """Every entry within rel * |b| + floor(n, G, ||H||_1)."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape
    fl = grad_floor(n, n_ops, h1)
    ok = np.abs(a - b) <= rel * np.abs(b) + fl
    return bool(np.all(ok))


def grad_report(a, b, n: int, n_ops: int, h1: float) -> str:
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    fl = grad_floor(n, n_ops, h1)
    d = np.abs(a - b)
    big = np.abs(b) > 1e3 * fl
    worst_rel = float(np.max(d[big] / np.abs(b[big]))) if np.any(big) else 0.0
    return (f"max|da|={float(d.max()):.3e} floor={fl:.3e} max rel (|b|>1e3 floor)={worst_rel:.3e} "
            f"max|b|={float(np.abs(b).max()):.3e}")
