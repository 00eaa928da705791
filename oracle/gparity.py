"""Wilson operator with G-parity boundary conditions (the paper lists
"G-parity boundary conditions" among its actions, Sec. 4, without a formula).

Reading (the standard two-flavour formulation): the field has two flavours,
Psi = (Psi_0, Psi_1) with Psi_1 the charge conjugate of the second quark
flavour, so flavour 1 couples to the complex-conjugate links U*. In every
G-parity direction mu the boundary twists flavour:

    Psi_0(x + L_mu mu_hat) = +Psi_1(x),     Psi_1(x + L_mu mu_hat) = -Psi_0(x),

replacing that direction's ordinary boundary phase; other directions keep
theirs. The operator is the Wilson one, D = (4 + m) - H / 2, with the hop

    (H Psi)_f(x) = sum_mu [ (1 - gamma_mu) U^(f)_mu(x) Psi~_f(x + mu)
                          + (1 + gamma_mu) U^(f')_mu(x - mu)^dag Psi~_f(x - mu) ],

where Psi~_f(x +- mu) is the neighbour seen through the twist (flavour f' =
1 - f and the sign above when the hop crosses a G-parity boundary, else f'
= f), U^(0) = U and U^(1) = U*. The forward link belongs to the site x
(flavour f), the backward link to the neighbour (flavour f').

With a single G-parity direction this is the ordinary Wilson operator on the
lattice doubled in that direction, with links U on the first copy and U* on
the second and an antiperiodic wrap of the doubled extent; the pins use that
(tests/test_oracle_gparity.py), with the free-field spectrum for several
twisted directions, gamma_5-hermiticity and gauge covariance.

Fields: psi[2, t, z, y, x, spin, colour] (flavour first), U[t, z, y, x, mu, 3, 3].
"""
from __future__ import annotations

import numpy as np

from . import wilson
from .gamma import one_minus_gamma, one_plus_gamma, spin_apply


def _flavour_links(u: np.ndarray) -> np.ndarray:
    """(U^(0), U^(1)) = (U, U*) stacked on a leading flavour axis."""
    return np.stack([u, np.conj(u)])


def _neighbour(psi2: np.ndarray, mu: int, sign: int, bc, twisted: bool) -> np.ndarray:
    """Psi~_f(x + sign mu) for both flavours: [2, t, z, y, x, 4, 3]."""
    ax = wilson.site_axis(mu)
    out = np.roll(psi2, -sign, axis=ax)
    L = psi2.shape[ax]
    edge = [slice(None)] * psi2.ndim
    edge[psi2.ndim + ax] = L - 1 if sign > 0 else 0
    edge = tuple(edge)
    if not twisted:
        if bc[mu] != 1.0:
            out[edge] *= bc[mu]
        return out
    wrapped = out[edge].copy()  # the neighbour's own flavour, read across the boundary
    s0, s1 = (1.0, -1.0) if sign > 0 else (-1.0, 1.0)
    f0 = (0,) + edge[1:]
    f1 = (1,) + edge[1:]
    out[f0] = s0 * wrapped[1]
    out[f1] = s1 * wrapped[0]
    return out


def _backward_links(U: np.ndarray, mu: int, twisted: bool) -> np.ndarray:
    """U^(f')_mu(x - mu) for both flavours: [2, t, z, y, x, 3, 3]."""
    u = U[..., mu, :, :]
    ax = wilson.site_axis(mu)
    ub = np.roll(u, 1, axis=ax)
    links = _flavour_links(ub)
    if twisted:
        edge = [slice(None)] * links.ndim
        edge[links.ndim + ax] = 0
        edge = tuple(edge)
        swapped = links[edge][::-1].copy()  # owner of the link is the other flavour
        links[edge] = swapped
    return links


def hop(U: np.ndarray, psi2: np.ndarray, bc, gdirs, dagger: bool = False) -> np.ndarray:
    out = np.zeros_like(psi2)
    for mu in range(4):
        tw = mu in gdirs
        pm, pp = (one_minus_gamma(mu), one_plus_gamma(mu)) if not dagger else (one_plus_gamma(mu), one_minus_gamma(mu))
        u = U[..., mu, :, :]
        uf = _flavour_links(u)  # forward link of flavour f: U^(f)_mu(x)
        fwd = _neighbour(psi2, mu, +1, bc, tw)
        out += spin_apply(pm, np.einsum("f...ab,f...sb->f...sa", uf, fwd))
        ub = _backward_links(U, mu, tw)
        bwd = _neighbour(psi2, mu, -1, bc, tw)
        out += spin_apply(pp, np.einsum("f...ba,f...sb->f...sa", np.conj(ub), bwd))
    return out


def dirac(U: np.ndarray, psi2: np.ndarray, mass: float, bc, gdirs, dagger: bool = False) -> np.ndarray:
    return (4.0 + mass) * psi2 - 0.5 * hop(U, psi2, bc, gdirs, dagger)
