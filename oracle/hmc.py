"""Hybrid Monte Carlo molecular-dynamics trajectory for the Wilson gauge action
plus one Wilson pseudofermion (the paper lists HMC, the Wilson gauge and
Wilson fermion actions and the leapfrog and minimum-norm integrators, Sec. 4;
the definitions are the textbook ones).

  H(U, P) = K(P) + S_g(U) + S_f(U),   K(P) = sum_links tr(P^2) / 2,
  S_f(U) = phi^dag (M^dag M)^-1 phi   (M = D_W, mass normalisation),
  dU/dt = i P U,   dP/dt = -F(U),  F = F_gauge + F_fermion, each traceless
  Hermitian with dS = eps tr(T F) for U -> exp(i eps T) U.

Integrators over nsteps steps of eps = tau / nsteps:
  leapfrog        P(eps/2) U(eps) P(eps) U(eps) ... U(eps) P(eps/2)
  minimum norm    per step P(lam eps) U(eps/2) P((1 - 2 lam) eps) U(eps/2) P(lam eps),
  (2nd order)     lam = 0.1931833275037836 (Omelyan, Mryglod and Folk, 2003);
where P(h): P <- P - h F(U) and U(h): U <- exp(i h P) U. Consecutive momentum
half-steps of neighbouring steps are merged. Accept / reject is left to the
caller (it needs a random number).

Momentum and pseudofermion refresh are the caller's: P with density
exp(-tr P^2 / 2) on traceless Hermitian matrices is what
synthetic.random_su3_algebra draws; phi = M^dag eta with eta of density
exp(-eta^dag eta) (re and im of each component N(0, 1/2)).

Pins (tests/test_oracle_hmc.py): reversibility, the O(eps^2) scaling of the
energy violation for both integrators, and exact energy conservation of each
sub-step's generator in the eps -> 0 limit.
"""
from __future__ import annotations

import numpy as np

from . import force as fermion_force
from . import gauge

LEAPFROG = 0
MINNORM2 = 1
LAMBDA_MN2 = 0.1931833275037836


def total_force(U, phi, mass, bc, beta, fermion=True, tol=1e-14):
    F = gauge.force(U, beta)
    if fermion:
        _, _, Ff, _, _ = fermion_force.force(U, phi, mass, bc, tol=tol)
        F = F + Ff
    return F


def hamiltonian(U, P, phi, mass, bc, beta, fermion=True, tol=1e-14):
    """(H, K, S_g, S_f)."""
    K = gauge.kinetic(P)
    Sg = gauge.action(U, beta)
    Sf = fermion_force.action(U, phi, mass, bc, fermion_force.solve_normal(U, phi, mass, bc, tol=tol)[0]) \
        if fermion else 0.0
    return K + Sg + Sf, K, Sg, Sf


def trajectory(U, P, phi, mass, bc, beta, tau, nsteps, integrator=LEAPFROG, fermion=True, tol=1e-14):
    """Integrate (U, P) over tau; returns (U1, P1, H0, H1, n_force)."""
    eps = tau / nsteps
    H0 = hamiltonian(U, P, phi, mass, bc, beta, fermion, tol)[0]
    U = U.copy()
    P = P.copy()
    nforce = 0

    def kick(h):
        nonlocal P, nforce
        P = P - h * total_force(U, phi, mass, bc, beta, fermion, tol)
        nforce += 1

    def drift(h):
        nonlocal U
        U = gauge.update_links(U, P, h)

    if integrator == LEAPFROG:
        kick(eps / 2)
        for k in range(nsteps):
            drift(eps)
            kick(eps if k < nsteps - 1 else eps / 2)
    elif integrator == MINNORM2:
        lam = LAMBDA_MN2
        kick(lam * eps)
        for k in range(nsteps):
            drift(eps / 2)
            kick((1 - 2 * lam) * eps)
            drift(eps / 2)
            kick(2 * lam * eps if k < nsteps - 1 else lam * eps)
    else:
        raise ValueError(integrator)
    H1 = hamiltonian(U, P, phi, mass, bc, beta, fermion, tol)[0]
    return U, P, H0, H1, nforce
