"""Conjugate gradient (Hestenes-Stiefel) for a Hermitian positive-definite A.

The paper lists "Conjugate gradient" among its algorithms (Sec. 4) and its
global reductions (Sec. 1) without writing the iteration down. Textbook form,
x_0 = 0:

  r = b, p = r, rr = <r, r>
  repeat: Ap = A p; alpha = rr / <p, Ap>; x += alpha p; r -= alpha Ap;
          rr' = <r, r>; beta = rr' / rr; p = r + beta p; rr = rr'
  until sqrt(rr / <b, b>) <= tol.

At exit the true residual ||b - A x|| / ||b|| is recomputed from x. A
multi-right-hand-side solve is defined column by column. Pinned against a
dense LU solve (tests/test_oracle_cg.py).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class CGInfo:
    iterations: int
    true_rel_residual: float
    converged: bool


def _dot(a: np.ndarray, b: np.ndarray) -> complex:
    return np.vdot(a.ravel(), b.ravel())


def cg(apply_a, b: np.ndarray, tol: float, maxiter: int):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = _dot(r, r).real
    bb = rr
    it = 0
    while it < maxiter and rr > tol * tol * bb:
        ap = apply_a(p)
        alpha = rr / _dot(p, ap).real
        x += alpha * p
        r -= alpha * ap
        rr_new = _dot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    true = true_residual(apply_a, x, b) if bb > 0 else 0.0
    return x, CGInfo(iterations=it, true_rel_residual=float(true), converged=bool(true <= tol))


def true_residual(apply_a, x: np.ndarray, b: np.ndarray) -> float:
    """||b - A x|| / ||b|| in FP64."""
    r = b - apply_a(x)
    return float(np.sqrt(_dot(r, r).real / _dot(b, b).real))
