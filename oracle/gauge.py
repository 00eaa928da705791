"""Wilson gauge action, its force, and the SU(3) link update of molecular dynamics.

The paper lists the "Wilson Gauge Action" and HMC among its actions and
algorithms (Sec. 4) without writing them down; these are the textbook
definitions, on the gauge field U[t, z, y, x, mu, 3, 3] with periodic
boundaries in every direction (fermion boundary phases do not enter here):

  plaquette   U_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  action      S_g = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3)
  staple      Sigma_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
                                           + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) ]
              so that the six plaquettes through U_mu(x) give Re tr(U_mu(x) Sigma_mu(x))
  force       for U_mu(x) -> exp(i eps T) U_mu(x), T traceless Hermitian,
              dS_g = eps tr(T F_mu(x)) with W = U_mu(x) Sigma_mu(x) and
              F_mu(x) = (beta / 3) * traceless part of (W - W^dag) / (2 i)
  update      U -> exp(i eps P) U, P traceless Hermitian (exact exponential
              through the eigendecomposition of P)
  kinetic     K(P) = sum_links tr(P^2) / 2

Pins (tests/test_oracle_gauge.py): unit links, a single twisted link in closed
form, gauge invariance, the force against central finite differences of S_g,
and the exponential against the series definition.
"""
from __future__ import annotations

import numpy as np

from . import wilson

PERIODIC = (1.0, 1.0, 1.0, 1.0)


def dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def _fwd(f: np.ndarray, mu: int) -> np.ndarray:
    """f(x + mu) for a field [t, z, y, x, a, b]."""
    return wilson.shift(f, mu, +1, PERIODIC)


def _bwd(f: np.ndarray, mu: int) -> np.ndarray:
    return wilson.shift(f, mu, -1, PERIODIC)


def plaquette_field(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    u_mu, u_nu = U[..., mu, :, :], U[..., nu, :, :]
    return u_mu @ _fwd(u_nu, mu) @ dag(_fwd(u_mu, nu)) @ dag(u_nu)


def mean_plaquette(U: np.ndarray) -> float:
    """Average of Re tr U_munu / 3 over sites and the six planes."""
    total = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            total += np.trace(plaquette_field(U, mu, nu), axis1=-2, axis2=-1).real.sum() / 3.0
    return float(total / (6 * np.prod(U.shape[:4])))


def action(U: np.ndarray, beta: float) -> float:
    n_plaq = 6 * int(np.prod(U.shape[:4]))
    return float(beta * n_plaq * (1.0 - mean_plaquette(U)))


def staple(U: np.ndarray, mu: int) -> np.ndarray:
    u_mu = U[..., mu, :, :]
    s = np.zeros_like(u_mu)
    for nu in range(4):
        if nu == mu:
            continue
        u_nu = U[..., nu, :, :]
        s += _fwd(u_nu, mu) @ dag(_fwd(u_mu, nu)) @ dag(u_nu)
        # lower staple: evaluate at x - nu the product U_nu(y+mu)^dag U_mu(y)^dag U_nu(y), y = x - nu
        low = dag(_fwd(u_nu, mu)) @ dag(u_mu) @ u_nu
        s += _bwd(low, nu)
    return s


def _traceless(m: np.ndarray) -> np.ndarray:
    tr = np.trace(m, axis1=-2, axis2=-1) / 3.0
    return m - tr[..., None, None] * np.eye(3)


def force(U: np.ndarray, beta: float) -> np.ndarray:
    """F with dS_g = eps sum tr(T F) under U -> exp(i eps T) U; shaped like U."""
    F = np.zeros_like(U)
    for mu in range(4):
        w = U[..., mu, :, :] @ staple(U, mu)
        F[..., mu, :, :] = (beta / 3.0) * _traceless((w - dag(w)) / 2j)
    return F


def expm_i(P: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps P) for Hermitian P[..., 3, 3]."""
    w, v = np.linalg.eigh(P)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * eps * w), v.conj())


def update_links(U: np.ndarray, P: np.ndarray, eps: float) -> np.ndarray:
    return expm_i(P, eps) @ U


def kinetic(P: np.ndarray) -> float:
    return float(0.5 * np.einsum("...ij,...ji->...", P, P).real.sum())
