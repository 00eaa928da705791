"""Pseudofermion action S = phi^dag (M^dag M)^-1 phi and its gauge-link gradient.

The paper lists HMC among its algorithms (Sec. 4) but gives no force formula;
this is the textbook derivation, written for M = D_W (mass normalisation):

  X = (M^dag M)^-1 phi,  Y = M X,  S = Re <phi, X>
  dS = -2 Re <Y, dM X>,  dM = -dH / 2   =>   dS = Re <Y, dH X>.

Only the two hops through link U_mu(x) depend on it; with the boundary phase
ph of that link (bc[mu] if x_mu = L_mu - 1, else 1):

  A = sum_spin  X(x+mu) ((1 - gamma_mu) Y(x))^dag        (3x3, colour outer product)
  B = sum_spin ((1 + gamma_mu) X(x)) Y(x+mu)^dag
  dS = ph Re[ tr(dU A) + tr(dU^dag B) ].

Two outputs are produced per link:

* ``grad``: the conjugate-Wirtinger gradient G with dS = Re sum conj(dU) G,
  i.e. G = ph (A^dag + B) (the convention torch.autograd uses for a real loss);
* ``F``: the traceless Hermitian force for the left perturbation
  U -> exp(i eps T) U, dS = eps tr(T F): with G2 = ph (U A - B U^dag),
  F = traceless part of i (G2 - G2^dag) / 2.

Pinned by central finite differences of S along random su(3) directions and
by gauge covariance F -> g F g^dag (tests/test_oracle_force.py).
"""
from __future__ import annotations

import numpy as np

from . import cg as cg_mod
from . import wilson
from .gamma import one_minus_gamma, one_plus_gamma, spin_apply


def solve_normal(U, phi, mass, bc, tol=1e-13, maxiter=100000):
    """X = (M^dag M)^-1 phi by the oracle CG on the full lattice."""
    x, info = cg_mod.cg(lambda v: wilson.dirac_dag_dirac(U, v, mass, bc), phi, tol, maxiter)
    return x, info


def action(U, phi, mass, bc, X=None):
    if X is None:
        X, _ = solve_normal(U, phi, mass, bc)
    return float(np.vdot(phi.ravel(), X.ravel()).real)


def _outer_spin_sum(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """sum_spin a_spin b_spin^dag for fields [..., spin, colour] -> [..., 3, 3]."""
    return np.einsum("...sa,...sb->...ab", a, b.conj())


def force_terms(U, X, Y, bc):
    """Per-link (grad, F), each shaped like U: (T, Z, Y, X, 4, 3, 3)."""
    grad = np.zeros_like(U)
    F = np.zeros_like(U)
    for mu in range(4):
        u = U[..., mu, :, :]
        # shift() folds the link's boundary phase into the neighbour field once.
        x_fwd = wilson.shift(X, mu, +1, bc)
        y_fwd = wilson.shift(Y, mu, +1, bc)
        a = _outer_spin_sum(x_fwd, spin_apply(one_minus_gamma(mu), Y))
        b = _outer_spin_sum(spin_apply(one_plus_gamma(mu), X), y_fwd)
        grad[..., mu, :, :] = np.conj(np.swapaxes(a, -1, -2)) + b
        g2 = u @ a - b @ np.conj(np.swapaxes(u, -1, -2))
        f = 0.5j * (g2 - np.conj(np.swapaxes(g2, -1, -2)))
        tr = np.trace(f, axis1=-2, axis2=-1) / 3.0
        F[..., mu, :, :] = f - tr[..., None, None] * np.eye(3)
    return grad, F


def force(U, phi, mass, bc, tol=1e-13):
    """(S, grad, F, X, Y) for S = phi^dag (M^dag M)^-1 phi."""
    X, _ = solve_normal(U, phi, mass, bc, tol=tol)
    Y = wilson.dirac(U, X, mass, bc)
    grad, F = force_terms(U, X, Y, bc)
    return action(U, phi, mass, bc, X), grad, F, X, Y
